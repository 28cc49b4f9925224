"""ctypes binding of libhfdib.so (the C ABI declared in include/hfdib.h).

Argument marshalling only: every step of the SIMPLE sweep runs in the CUDA
kernels of the library.  PyTorch provides device memory and the stream.  The
library must have been built (paper_2606_06135_gb300.build); there is no
fallback -- load_library() raises when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "lib", "libhfdib.so")

LAMINAR, KEPSILON, KOMEGA_SST, KOMEGA, REALIZABLE_KE = 0, 1, 2, 3, 4
MODELS = {"laminar": LAMINAR, "kepsilon": KEPSILON, "komegasst": KOMEGA_SST, "komega": KOMEGA,
          "realizableke": REALIZABLE_KE}
BC_KIND = {"inlet": 0, "outlet": 1, "slip": 2, "wall": 3, "empty": 4}
SIDES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")
FIELDS = {"ux": 0, "uy": 1, "uz": 2, "p": 3, "k": 4, "eps": 5, "omega": 6, "nut": 7,
          "phix": 8, "phiy": 9, "phiz": 10}
RES_NAMES = ("Ux", "Uy", "Uz", "p", "epsw", "k", "cont", "p_iters", "n_lam", "n_switch")
NRES = 10
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "out of memory",
          -4: "not converged", -5: "diverged", -6: "state mismatch", -7: "too large", -8: "timeout"}

OBJECTIVES = {"pressure_drop": 0, "drag": 1}
PRESSURE_PHASES = ("start", "build0", "coarsen", "r0", "vc_smooth0", "vc_restrict", "vc_smooth", "vc_tail",
                   "vc_prolong", "vc_upsmooth", "vc_final", "cg_product", "cg_update", "end",
                   "b0_r0_share", "b0_tail_table", "b0_tail_level", "b0_tail_in", "b0_tail_done",
                   "b0_tail_down", "b0_tail_coarse", "b0_tail_up", "b0_loop", "b0_part")
WALL_SIDES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")

ERR_NOT_CONVERGED = -4
STATUS_TOO_LARGE = -7
ERR_TIMEOUT = -8


class HfdibError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s: %s (%d)" % (where, STATUS.get(code, "error"), code))
        self.code = code


class Tune(C.Structure):
    _fields_ = [("threads", C.c_int32), ("tail_cells", C.c_int32), ("coarse_sweeps", C.c_int32),
                ("us_per_sweep", C.c_double), ("candidates", C.c_int32)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double)]


class Bc(C.Structure):
    _fields_ = [("face", C.c_int32 * 6), ("u_in", C.c_double * 3), ("I_in", C.c_double),
                ("lt_in", C.c_double), ("p_out", C.c_double), ("u_ref", C.c_double),
                ("l_ref", C.c_double), ("u_s", C.c_double * 3)]


class Options(C.Structure):
    _fields_ = [("urf_u", C.c_double), ("urf_p", C.c_double), ("urf_turb", C.c_double),
                ("n_u", C.c_int32), ("n_turb", C.c_int32), ("p_reltol", C.c_double),
                ("p_maxiter", C.c_int32), ("precision", C.c_int32), ("precond", C.c_int32),
                ("p_check", C.c_int32), ("mg_coarse_sweeps", C.c_int32), ("graph", C.c_int32),
                ("p_persistent", C.c_int32), ("freeze_switch", C.c_int32), ("frozen_turbulence", C.c_int32),
                ("wall_distance", C.c_int32), ("continuity_mask", C.c_int32), ("convection", C.c_int32),
                ("mg_tail_cells", C.c_int32), ("p_cg32", C.c_int32)]


_LIB = None

# hfdib_alloc_fn / hfdib_free_fn of include/hfdib.h
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_ALLOCATOR = None     # the installed callbacks (kept alive while installed)

EXPORTED = ("hfdib_default_options", "hfdib_create", "hfdib_simple_sweep", "hfdib_solve_steady",
            "hfdib_get_field", "hfdib_set_field", "hfdib_get_tags", "hfdib_get_bc_list",
            "hfdib_get_history", "hfdib_get_state", "hfdib_set_state", "hfdib_get_counters",
            "hfdib_error_string", "hfdib_destroy", "hfdib_profile_sweeps", "hfdib_get_launch_counts",
            "hfdib_classify_noalloc", "hfdib_create_batch", "hfdib_batch_sweep", "hfdib_batch_solve_steady",
            "hfdib_batch_handle", "hfdib_batch_autotune", "hfdib_destroy_batch", "hfdib_adjoint_grad",
            "hfdib_ib_force", "hfdib_wall_shear", "hfdib_recirculation", "hfdib_set_barrier_polls",
            "hfdib_batch_set_barrier_polls", "hfdib_force_coefficients", "hfdib_pressure_trace",
            "hfdib_set_allocator")
KERNEL_CLASSES = ("imposed", "grad_u", "mom_asm", "mom_smooth", "hbya", "p_coef", "pcg", "vcycle0",
                  "update", "turb_prep", "scal_asm", "scal_smooth", "turb_final", "sweep_end")


def load_library(path=LIBPATH):
    """Load libhfdib.so once and declare the C signatures."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError("libhfdib.so not built (%s); run paper_2606_06135_gb300.build" % path)
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    lib.hfdib_default_options.argtypes = [C.POINTER(Options)]
    lib.hfdib_default_options.restype = None
    lib.hfdib_create.argtypes = [C.POINTER(Grid), vp, vp, i32, dbl, C.POINTER(Bc), C.POINTER(Options),
                                 vp, C.POINTER(vp)]
    lib.hfdib_simple_sweep.argtypes = [vp, i32, vp]
    lib.hfdib_solve_steady.argtypes = [vp, dbl, i32, i32, C.POINTER(i32), vp]
    lib.hfdib_get_field.argtypes = [vp, i32, vp]
    lib.hfdib_set_field.argtypes = [vp, i32, vp]
    lib.hfdib_get_tags.argtypes = [vp, vp, C.POINTER(i64)]
    lib.hfdib_get_bc_list.argtypes = [vp, vp, vp, vp]
    lib.hfdib_get_history.argtypes = [vp, i32, vp, C.POINTER(i32)]
    lib.hfdib_get_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    lib.hfdib_set_state.argtypes = [vp, vp, C.c_size_t]
    lib.hfdib_get_counters.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    lib.hfdib_profile_sweeps.argtypes = [vp, i32, vp, vp, i32]
    lib.hfdib_profile_sweeps.restype = C.c_int
    lib.hfdib_get_launch_counts.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    lib.hfdib_get_launch_counts.restype = C.c_int
    lib.hfdib_classify_noalloc.argtypes = [C.POINTER(Grid), vp, vp, vp, i64, C.POINTER(i64), vp]
    lib.hfdib_classify_noalloc.restype = C.c_int
    lib.hfdib_create_batch.argtypes = [i32, vp, vp, vp, i32, vp, vp, C.POINTER(Options), vp, C.POINTER(vp)]
    lib.hfdib_create_batch.restype = C.c_int
    lib.hfdib_batch_sweep.argtypes = [vp, i32, vp]
    lib.hfdib_batch_sweep.restype = C.c_int
    lib.hfdib_batch_solve_steady.argtypes = [vp, dbl, i32, i32, vp, vp]
    lib.hfdib_batch_solve_steady.restype = C.c_int
    lib.hfdib_batch_handle.argtypes = [vp, i32, C.POINTER(vp)]
    lib.hfdib_batch_handle.restype = C.c_int
    lib.hfdib_batch_autotune.argtypes = [vp, i32, C.POINTER(Tune)]
    lib.hfdib_batch_autotune.restype = C.c_int
    lib.hfdib_destroy_batch.argtypes = [vp]
    lib.hfdib_destroy_batch.restype = None
    lib.hfdib_adjoint_grad.argtypes = [vp, i32, dbl, i32, i32, vp, C.POINTER(dbl), C.POINTER(i32), C.POINTER(dbl)]
    lib.hfdib_adjoint_grad.restype = i32
    lib.hfdib_ib_force.argtypes = [vp, vp]
    lib.hfdib_ib_force.restype = i32
    lib.hfdib_wall_shear.argtypes = [vp, i32, vp, C.POINTER(i64)]
    lib.hfdib_wall_shear.restype = i32
    lib.hfdib_recirculation.argtypes = [vp, dbl, vp]
    lib.hfdib_recirculation.restype = i32
    lib.hfdib_force_coefficients.argtypes = [vp, dbl, dbl, vp]
    lib.hfdib_force_coefficients.restype = i32
    lib.hfdib_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    lib.hfdib_set_allocator.restype = i32
    lib.hfdib_pressure_trace.argtypes = [vp, vp, i32, C.POINTER(i32)]
    lib.hfdib_pressure_trace.restype = i32
    lib.hfdib_set_barrier_polls.argtypes = [vp, i64]
    lib.hfdib_set_barrier_polls.restype = i32
    lib.hfdib_batch_set_barrier_polls.argtypes = [vp, i64]
    lib.hfdib_batch_set_barrier_polls.restype = i32
    lib.hfdib_error_string.argtypes = [i32]
    lib.hfdib_error_string.restype = C.c_char_p
    lib.hfdib_destroy.argtypes = [vp]
    lib.hfdib_destroy.restype = None
    for name in EXPORTED:
        f = getattr(lib, name)
        if f.restype is C.c_int or name in ("hfdib_create", "hfdib_simple_sweep", "hfdib_solve_steady",
                                             "hfdib_get_field", "hfdib_set_field", "hfdib_get_tags",
                                             "hfdib_get_bc_list", "hfdib_get_history", "hfdib_get_state",
                                             "hfdib_set_state", "hfdib_get_counters"):
            f.restype = C.c_int
    _LIB = lib
    return lib


def use_torch_allocator():
    """Device memory of the handles and batches created from now on comes from
    PyTorch's caching allocator (hfdib_set_allocator): blocks are allocated
    on the handle's stream and returned at destroy."""
    global _ALLOCATOR
    if _ALLOCATOR is not None and _ALLOCATOR[0] == "torch":
        return
    import torch
    lib = load_library()

    def alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
        except Exception:
            return None        # out of memory: the library reports HFDIB_ERR_OOM

    def free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    cbs = ("torch", ALLOC_FN(alloc), FREE_FN(free))
    _check(lib.hfdib_set_allocator(cbs[1], cbs[2], None), "hfdib_set_allocator")
    _ALLOCATOR = cbs


def use_cuda_malloc():
    """Handles and batches created from now on allocate with cudaMalloc."""
    global _ALLOCATOR
    lib = load_library()
    _check(lib.hfdib_set_allocator(ALLOC_FN(), FREE_FN(), None), "hfdib_set_allocator")
    # the old callbacks may still serve handles made while they were installed
    if _ALLOCATOR is not None:
        _RETIRED.append(_ALLOCATOR)
    _ALLOCATOR = ("cuda", None, None)


_RETIRED = []


def default_options(**kw):
    lib = load_library()
    o = Options()
    lib.hfdib_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _check(rc, where):
    if rc != 0:
        raise HfdibError(rc, where)


def grid_struct(g):
    return Grid(g["nx"], g["ny"], g["nz"], g["x0"], g["y0"], g["z0"], g["dx"], g["dy"], g["dz"])


def bc_struct(case):
    b = Bc()
    for s, name in enumerate(SIDES):
        b.face[s] = BC_KIND[case["bc"][name]]
    for q in range(3):
        b.u_in[q] = case["u_in"][q]
        b.u_s[q] = case["u_s"][q]
    b.I_in = case["I_in"]
    b.lt_in = case["lt_in"]
    b.p_out = case["p_out"]
    b.u_ref = case["u_ref"]
    b.l_ref = case["l_ref"]
    return b


class Solver:
    """One HFDIB steady-RANS problem on the GPU (wraps one hfdib handle)."""

    def __init__(self, case, device="cuda:0", stream=None, **opts):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.case = case
        self.device = torch.device(device)
        g = case["grid"]
        self.shape = (g["nz"], g["ny"], g["nx"])
        self.N = g["nx"] * g["ny"] * g["nz"]
        self.dims = 2 if g["nz"] == 1 else 3
        self.face_counts = ((g["nx"] + 1) * g["ny"] * g["nz"], g["nx"] * (g["ny"] + 1) * g["nz"],
                            g["nx"] * g["ny"] * (g["nz"] + 1))
        self.model = MODELS[case["model"]]
        # a dedicated stream: sweeps are captured as CUDA graphs, which the
        # legacy default stream does not allow
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        def dev_array(x):
            if x is None:
                return None
            if isinstance(x, torch.Tensor):
                return x.to(self.device, torch.float64).contiguous()
            return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).to(self.device)
        lam = dev_array(case["lam"])
        yw = dev_array(case.get("ywall"))
        torch.cuda.synchronize(self.device)
        if _ALLOCATOR is None:
            use_torch_allocator()
        self._opts = default_options(**opts)
        h = C.c_void_p()
        rc = self.lib.hfdib_create(C.byref(grid_struct(g)), C.c_void_p(lam.data_ptr()),
                                   C.c_void_p(yw.data_ptr()) if yw is not None else None,
                                   self.model, float(case["Re"]), C.byref(bc_struct(case)),
                                   C.byref(self._opts), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _check(rc, "hfdib_create")
        self.h = h

    # ------------------------------------------------------------------ sweeps
    def sweep(self, n=1, read=True):
        res = np.zeros(NRES) if read else None
        rc = self.lib.hfdib_simple_sweep(self.h, int(n), res.ctypes.data if read else None)
        _check(rc, "hfdib_simple_sweep")
        return res

    def pressure_trace(self, capacity=4096):
        """One sweep with the persistent pressure kernel's phase trace:
        a list of (phase name, ns since the kernel started)."""
        buf = np.zeros(2 * capacity, dtype=np.int64)
        n = C.c_int(0)
        self.stream.synchronize()
        _check(self.lib.hfdib_pressure_trace(self.h, buf.ctypes.data, int(capacity), C.byref(n)),
               "hfdib_pressure_trace")
        pairs = buf[: 2 * n.value].reshape(-1, 2)
        t0 = pairs[0, 1] if len(pairs) else 0
        return [(PRESSURE_PHASES[int(t)], int(ns - t0)) for t, ns in pairs]

    def set_barrier_polls(self, polls=0):
        """Poll budget of each wait at the persistent pressure kernel's grid
        barrier (0: the default); a wait that runs out makes the next
        residual read return HFDIB_ERR_TIMEOUT."""
        _check(self.lib.hfdib_set_barrier_polls(self.h, int(polls)), "hfdib_set_barrier_polls")

    def solve(self, tol=1e-6, max_iter=1000, check_every=10, raise_on_fail=False):
        it = C.c_int(0)
        res = np.zeros(NRES)
        rc = self.lib.hfdib_solve_steady(self.h, float(tol), int(max_iter), int(check_every),
                                         C.byref(it), res.ctypes.data)
        if rc not in (0, ERR_NOT_CONVERGED) or (raise_on_fail and rc != 0):
            _check(rc, "hfdib_solve_steady")
        return rc, it.value, res

    # ------------------------------------------------------------------ data
    def field(self, name):
        torch = self.torch
        fid = FIELDS[name]
        n = self.face_counts[fid - 8] if fid >= 8 else self.N
        out = torch.empty(n, dtype=torch.float64, device=self.device)
        _check(self.lib.hfdib_get_field(self.h, fid, C.c_void_p(out.data_ptr())), "hfdib_get_field")
        self.stream.synchronize()
        return out

    def set_field(self, name, values):
        torch = self.torch
        t = torch.as_tensor(values, dtype=torch.float64).to(self.device).contiguous().reshape(-1)
        fid = FIELDS[name]
        self.stream.synchronize()
        _check(self.lib.hfdib_set_field(self.h, fid, C.c_void_p(t.data_ptr())), "hfdib_set_field")
        self.stream.synchronize()

    def fields(self):
        names = ["ux", "uy", "uz"][: self.dims] + ["p", "nut"]
        if self.model != LAMINAR:
            names += ["k", "eps", "omega"]
        return {n: self.field(n).cpu().numpy().reshape(self.shape) for n in names}

    def tags(self):
        torch = self.torch
        t = torch.empty(self.N, dtype=torch.uint8, device=self.device)
        nbc = C.c_int64(0)
        _check(self.lib.hfdib_get_tags(self.h, C.c_void_p(t.data_ptr()), C.byref(nbc)), "hfdib_get_tags")
        return t.cpu().numpy().reshape(self.shape), nbc.value

    def bc_list(self):
        torch = self.torch
        _, nbc = self.tags()
        ints = torch.zeros((max(nbc, 1), 8), dtype=torch.int64, device=self.device)
        ints2 = torch.zeros((max(nbc, 1), 3), dtype=torch.int64, device=self.device)
        reals = torch.zeros((max(nbc, 1), 14), dtype=torch.float64, device=self.device)
        _check(self.lib.hfdib_get_bc_list(self.h, C.c_void_p(ints.data_ptr()), C.c_void_p(ints2.data_ptr()),
                                          C.c_void_p(reals.data_ptr())), "hfdib_get_bc_list")
        self.stream.synchronize()
        a = ints.cpu().numpy()[:nbc]
        a2 = ints2.cpu().numpy()[:nbc]
        r = reals.cpu().numpy()[:nbc]
        return dict(cell=a[:, 0], nbr=a[:, 1], case=a[:, 2], clamped=a[:, 3].astype(bool),
                    base1=a[:, 4:7], base2=a2, laminar=a[:, 7].astype(bool), n=r[:, 0:3], y_perp=r[:, 3], y_eff=r[:, 4],
                    wS=r[:, 5], w1=r[:, 6], w2=r[:, 7], t1=r[:, 8:11], t2=r[:, 11:14])

    def history(self, count=1024):
        buf = np.zeros((count, NRES))
        n = C.c_int(0)
        _check(self.lib.hfdib_get_history(self.h, int(count), buf.ctypes.data, C.byref(n)), "hfdib_get_history")
        return buf[: n.value]

    def counters(self):
        s, l = C.c_int64(0), C.c_int64(0)
        _check(self.lib.hfdib_get_counters(self.h, C.byref(s), C.byref(l)), "hfdib_get_counters")
        return s.value, l.value

    def profile(self, n_sweeps=3):
        """Per kernel class: (total device microseconds, timed launch groups)."""
        k = len(KERNEL_CLASSES)
        us = np.zeros(k)
        calls = np.zeros(k, dtype=np.int64)
        _check(self.lib.hfdib_profile_sweeps(self.h, int(n_sweeps), us.ctypes.data, calls.ctypes.data, k),
               "hfdib_profile_sweeps")
        return {name: (float(us[i]), int(calls[i])) for i, name in enumerate(KERNEL_CLASSES)}

    def launch_counts(self):
        """(launches per sweep outside the pressure loop, launches per pressure iteration)."""
        a, b = C.c_int64(0), C.c_int64(0)
        _check(self.lib.hfdib_get_launch_counts(self.h, C.byref(a), C.byref(b)), "hfdib_get_launch_counts")
        return a.value, b.value

    def adjoint_grad(self, tol=1e-10, max_iter=20000, objective="pressure_drop", gmres_restart=0):
        """Frozen-turbulence adjoint of the converged state: returns (J,
        dJ/dlambda as a device tensor shaped like lambda, transposed sweeps,
        final relative residual (GMRES) or change (gmres_restart=0: plain
        reverse fixed point), status).  Status 0, or -4 when max_iter ran out."""
        torch = self.torch
        out = torch.zeros(self.N, dtype=torch.float64, device=self.device)
        J = C.c_double(0.0)
        it = C.c_int(0)
        ch = C.c_double(0.0)
        self.stream.synchronize()
        objective = OBJECTIVES.get(objective, objective)
        rc = self.lib.hfdib_adjoint_grad(self.h, int(objective), float(tol), int(max_iter), int(gmres_restart),
                                         C.c_void_p(out.data_ptr()), C.byref(J), C.byref(it), C.byref(ch))
        if rc not in (0, ERR_NOT_CONVERGED):
            _check(rc, "hfdib_adjoint_grad")
        self.stream.synchronize()
        return J.value, out.reshape(self.shape), it.value, ch.value, rc

    def objective(self, objective="pressure_drop"):
        """J of the current state (hfdib_adjoint_grad with max_iter = 0)."""
        objective = OBJECTIVES.get(objective, objective)
        J = C.c_double(0.0)
        self.stream.synchronize()
        rc = self.lib.hfdib_adjoint_grad(self.h, int(objective), 1.0, 0, 0, None, C.byref(J), None, None)
        _check(rc, "hfdib_adjoint_grad")
        return J.value

    # ------------------------------------------------------------------ forces
    def force(self):
        """Force of the fluid on the body (hfdib_ib_force): (pressure part,
        viscous and convective part), each a length-3 numpy array."""
        out = np.zeros(6)
        self.stream.synchronize()
        _check(self.lib.hfdib_ib_force(self.h, out.ctypes.data), "hfdib_ib_force")
        return out[:3].copy(), out[3:].copy()

    def force_coefficients(self, A_ref=None, gamma=0.0):
        """(C_d, C_l) of Eqs. dragcoeff and dlcoeffs (hfdib_force_coefficients).
        A_ref None: l_ref times the cell depth dz (2D grids)."""
        out = np.zeros(2)
        self.stream.synchronize()
        _check(self.lib.hfdib_force_coefficients(self.h, 0.0 if A_ref is None else float(A_ref), float(gamma),
                                                 out.ctypes.data), "hfdib_force_coefficients")
        return float(out[0]), float(out[1])

    def wall_shear(self, side):
        """tau_w along a no-slip domain side ('ymin', ...): device tensor
        [3, n_faces] (hfdib_wall_shear)."""
        torch = self.torch
        sid = WALL_SIDES.index(side) if isinstance(side, str) else int(side)
        nf = C.c_int64(0)
        _check(self.lib.hfdib_wall_shear(self.h, sid, None, C.byref(nf)), "hfdib_wall_shear")
        out = torch.empty((3, nf.value), dtype=torch.float64, device=self.device)
        self.stream.synchronize()
        _check(self.lib.hfdib_wall_shear(self.h, sid, C.c_void_p(out.data_ptr()), None), "hfdib_wall_shear")
        self.stream.synchronize()
        return out

    def recirculation(self, x_rear):
        """(length, volume, cells) of the region behind x_rear with u_x < 0
        (hfdib_recirculation)."""
        out = np.zeros(3)
        self.stream.synchronize()
        _check(self.lib.hfdib_recirculation(self.h, float(x_rear), out.ctypes.data), "hfdib_recirculation")
        return float(out[0]), float(out[1]), int(out[2])

    def get_state(self):
        n = C.c_size_t(0)
        _check(self.lib.hfdib_get_state(self.h, None, C.byref(n)), "hfdib_get_state")
        buf = np.zeros(n.value, dtype=np.uint8)
        _check(self.lib.hfdib_get_state(self.h, buf.ctypes.data, C.byref(n)), "hfdib_get_state")
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(self.lib.hfdib_set_state(self.h, buf.ctypes.data, buf.nbytes), "hfdib_set_state")

    @classmethod
    def view(cls, handle, case, device, stream, lib):
        """Field access to a problem owned by a batch (does not own the handle)."""
        self = cls.__new__(cls)
        import torch
        self.torch = torch
        self.lib = lib
        self.case = case
        self.device = torch.device(device)
        g = case["grid"]
        self.shape = (g["nz"], g["ny"], g["nx"])
        self.N = g["nx"] * g["ny"] * g["nz"]
        self.dims = 2 if g["nz"] == 1 else 3
        self.face_counts = ((g["nx"] + 1) * g["ny"] * g["nz"], g["nx"] * (g["ny"] + 1) * g["nz"],
                            g["nx"] * g["ny"] * (g["nz"] + 1))
        self.model = MODELS[case["model"]]
        self.stream = stream
        self.h = handle
        self.owned = False
        return self

    def close(self):
        if getattr(self, "h", None) and getattr(self, "owned", True):
            self.lib.hfdib_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """B independent problems advanced together (one batched persistent
    pressure launch per sweep, the sweep captured as one CUDA graph)."""

    def __init__(self, cases, device="cuda:0", stream=None, **opts):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.cases = list(cases)
        self.B = len(self.cases)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        models = {c["model"] for c in self.cases}
        if len(models) != 1:
            raise ValueError("a batch shares one turbulence model")
        model = MODELS[models.pop()]

        def dev(x):
            if x is None:
                return None
            if isinstance(x, torch.Tensor):
                return x.to(self.device, torch.float64).contiguous()
            return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).to(self.device)
        self._lam = [dev(c["lam"]) for c in self.cases]
        self._yw = [dev(c.get("ywall")) for c in self.cases]
        torch.cuda.synchronize(self.device)
        if _ALLOCATOR is None:
            use_torch_allocator()
        B = self.B
        grids = (Grid * B)(*[grid_struct(c["grid"]) for c in self.cases])
        bcs = (Bc * B)(*[bc_struct(c) for c in self.cases])
        re = (C.c_double * B)(*[float(c["Re"]) for c in self.cases])
        lam = (C.c_void_p * B)(*[t.data_ptr() for t in self._lam])
        yw = (C.c_void_p * B)(*[(t.data_ptr() if t is not None else None) for t in self._yw])
        self._opts = default_options(**opts)
        h = C.c_void_p()
        rc = self.lib.hfdib_create_batch(B, grids, lam, yw, model, re, bcs, C.byref(self._opts),
                                         C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _check(rc, "hfdib_create_batch")
        self.h = h

    def sweep(self, n=1, read=True):
        res = np.zeros((self.B, NRES)) if read else None
        _check(self.lib.hfdib_batch_sweep(self.h, int(n), res.ctypes.data if read else None), "hfdib_batch_sweep")
        return res

    def solve(self, tol=1e-6, max_iter=1000, check_every=10):
        it = np.zeros(self.B, dtype=np.int32)
        res = np.zeros((self.B, NRES))
        rc = self.lib.hfdib_batch_solve_steady(self.h, float(tol), int(max_iter), int(check_every),
                                               it.ctypes.data, res.ctypes.data)
        if rc not in (0, ERR_NOT_CONVERGED):
            _check(rc, "hfdib_batch_solve_steady")
        return rc, it, res

    def set_barrier_polls(self, polls=0):
        _check(self.lib.hfdib_batch_set_barrier_polls(self.h, int(polls)), "hfdib_batch_set_barrier_polls")

    def problem(self, i):
        hh = C.c_void_p()
        _check(self.lib.hfdib_batch_handle(self.h, int(i), C.byref(hh)), "hfdib_batch_handle")
        return Solver.view(hh, self.cases[i], self.device, self.stream, self.lib)

    def autotune(self, trial_sweeps=2):
        t = Tune()
        _check(self.lib.hfdib_batch_autotune(self.h, int(trial_sweeps), C.byref(t)), "hfdib_batch_autotune")
        return dict(threads=t.threads, tail_cells=t.tail_cells, coarse_sweeps=t.coarse_sweeps,
                    us_per_sweep=t.us_per_sweep, candidates=t.candidates)

    def close(self):
        if getattr(self, "h", None):
            self.lib.hfdib_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
