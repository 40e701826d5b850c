"""GB300 (sm_103a) implementation of the RBF neural-field hot path of Shaw,
Kilpatrick & Avitabile, "Radial Basis Function Techniques for Neural Field Models on
Surfaces".

This module is a thin ctypes binding over the C-ABI library ``libnf.so``
(declared in ``include/nf.h``).  It only marshals torch CUDA tensors (pointers,
sizes, the current stream) into those calls; every step of the computation runs in
the library's CUDA kernels.  If the library is missing or cannot be loaded, every
entry point raises -- there is no CPU fallback.

Entry points (same names as the C ABI):

* :func:`nf_build_stencils`  §3.1 stencils S(E)
* :func:`nf_quad_weights`    §3.2 Eq. (3.5) / §3.3 Eq. (3.6) quadrature weights
* :class:`Operator`          W diag(q) of Eq. (2.9): ``nf_operator_create``
* :func:`nf_nonlocal_apply`  I = sum_j w(x_i, x_j) q_j f(u_j)
* :func:`nf_rk4_advance`     RK4 on Eq. (2.9)
* :func:`nf_adjoint`         discrete adjoint of the RK4 map
* :class:`NeuralFieldRK4`    autograd Function: RK4 forward, adjoint backward
* :func:`nf_mms_sphere_eigs` Funk-Hecke eigenvalues for manufactured forcing
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import _build

__all__ = [
    "NFError", "lib", "build", "nf_build_stencils", "nf_quad_weights", "Operator", "nf_nonlocal_apply",
    "nf_rk4_advance", "nf_adjoint", "nf_mms_sphere_eigs", "Forcing", "MATRIX_FREE", "DENSE_FP32",
    "DENSE_BF16X2", "DENSE_SYM_FP32", "DENSE_SYM_BF16X2", "STATUS", "nf_field_advance", "MODEL_FIELD", "MODEL_DEPRESSION",
    "RATE_SIGMOID", "RATE_SMOOTHSTEP", "FORCE_NONE", "FORCE_MMS_EIGEN", "FORCE_MMS_FLAT", "FORCE_MMS_SPHERE",
    "NeuralFieldRK4", "nf_build_stencils_at",
    "MF_AUTO", "MF_SYMMETRIC", "MF_PACKED", "MF_SYMMETRIC_512", "MF_SYMMETRIC_1024",
]

MATRIX_FREE, DENSE_FP32, DENSE_BF16X2, DENSE_SYM_FP32, DENSE_SYM_BF16X2 = 0, 1, 2, 4, 5
FORCE_NONE, FORCE_MMS_EIGEN, FORCE_MMS_FLAT, FORCE_MMS_SPHERE = 0, 1, 2, 3
MF_AUTO, MF_SYMMETRIC, MF_PACKED, MF_SYMMETRIC_512, MF_SYMMETRIC_1024 = 0, 1, 2, 3, 4
STATUS = {0: "NF_OK", 1: "NF_ERR_ARG", 2: "NF_ERR_SINGULAR", 3: "NF_ERR_NONFINITE", 4: "NF_ERR_TIMEOUT",
          5: "NF_ERR_NOMEM", 6: "NF_ERR_CUDA", 7: "NF_ERR_UNSUPPORTED"}

# exported symbols declared in include/nf.h
EXPORTS = ["nf_last_error", "nf_version", "nf_build_stencils", "nf_quad_weights", "nf_operator_create",
           "nf_operator_destroy", "nf_operator_check", "nf_nonlocal_apply", "nf_mms_sphere_eigs",
           "nf_rk4_advance", "nf_adjoint", "nf_operator_profile", "nf_operator_kernel_ms",
           "nf_nonlocal_apply_noalloc", "nf_operator_group", "nf_operator_launch_shape", "nf_selftest_timeout",
           "nf_operator_mf_schedule", "nf_operator_mf_cull", "nf_field_advance", "nf_noalloc_status",
           "nf_noalloc_limits", "nf_selftest_noalloc_flag", "nf_operator_kernel_ms_history",
           "nf_probe_pipe", "nf_operator_group_tuning", "nf_operator_group_configure", "nf_build_stencils_at",
           "nf_quad_weights_opts"]


class NFError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


class _Kernel(C.Structure):
    _fields_ = [("A1", C.c_float), ("s1", C.c_float), ("A2", C.c_float), ("s2", C.c_float), ("period", C.c_float)]


class _Model(C.Structure):
    _fields_ = [("kind", C.c_int), ("rate", C.c_int), ("a", C.c_float), ("b", C.c_float), ("tau", C.c_float),
                ("beta_d", C.c_float)]


class _QuadOpts(C.Structure):
    _fields_ = [("dim", C.c_int), ("phs_order", C.c_int), ("poly_deg", C.c_int), ("curved", C.c_int)]


class _Forcing(C.Structure):
    _fields_ = [("kind", C.c_int), ("Y1", C.c_void_p), ("Y2", C.c_void_p), ("c", C.c_double),
                ("a0", C.c_double), ("lam0", C.c_double), ("lam1", C.c_double), ("lam2", C.c_double),
                ("radius", C.c_double), ("sigma", C.c_double), ("scale", C.c_double)]


_lib = None
_vp = C.c_void_p
_i64 = C.c_int64


def build(force: bool = False) -> str:
    return _build.build(force=force)


def lib(path: str | None = None):
    """Load ``libnf.so`` (building it if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not found at {path}")
    L = C.CDLL(path)
    L.nf_last_error.restype = C.c_char_p
    L.nf_version.restype = C.c_int
    for name in EXPORTS[2:]:
        getattr(L, name).restype = C.c_int
    L.nf_build_stencils.argtypes = [_vp, _i64, C.c_int, _vp, _i64, C.c_int, _vp, _vp]
    L.nf_build_stencils_at.argtypes = [_vp, _i64, C.c_int, _vp, _i64, C.c_int, _vp, _vp]
    L.nf_quad_weights_opts.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, C.c_int, C.POINTER(_QuadOpts), _vp,
                                       C.POINTER(C.c_int64), _vp]
    L.nf_quad_weights.argtypes = [_vp, _vp, _i64, C.c_int, _vp, _i64, _vp, C.c_int, C.c_int, _vp,
                                  C.POINTER(C.c_int64), _vp]
    L.nf_operator_create.argtypes = [_vp, _vp, _i64, _Kernel, C.c_int, _vp, C.POINTER(_vp)]
    L.nf_operator_destroy.argtypes = [_vp]
    L.nf_operator_group.argtypes = [C.POINTER(_vp), C.POINTER(C.c_int), C.c_int, _vp, C.POINTER(_vp)]
    L.nf_operator_group_tuning.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                           C.POINTER(C.c_int), C.POINTER(C.c_float)]
    L.nf_operator_group_configure.argtypes = [_vp, C.c_int, C.c_int, C.c_double, _vp]
    L.nf_operator_check.argtypes = [_vp, _vp]
    L.nf_operator_profile.argtypes = [_vp, C.c_int]
    L.nf_operator_kernel_ms.argtypes = [_vp, C.POINTER(C.c_float)]
    L.nf_operator_kernel_ms_history.argtypes = [_vp, C.c_int, C.POINTER(C.c_float)]
    L.nf_operator_launch_shape.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.nf_operator_mf_schedule.argtypes = [_vp, C.c_int]
    L.nf_operator_mf_cull.argtypes = [_vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _vp]
    L.nf_selftest_timeout.argtypes = [_vp]
    L.nf_nonlocal_apply.argtypes = [_vp, _vp, C.c_int, _vp, _vp, _vp, _vp]
    L.nf_nonlocal_apply_noalloc.argtypes = [_vp, _vp, _i64, _Kernel, _vp, C.c_float, C.c_float, _vp, _vp]
    L.nf_noalloc_status.argtypes = [_vp]
    L.nf_noalloc_limits.argtypes = [_i64, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.nf_selftest_noalloc_flag.argtypes = [_i64, _vp, _vp]
    L.nf_probe_pipe.argtypes = [C.c_int, _i64, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_float),
                                _vp]
    L.nf_mms_sphere_eigs.argtypes = [_Kernel, C.POINTER(C.c_double)]
    L.nf_rk4_advance.argtypes = [_vp, _vp, C.c_int, C.c_double, C.c_double, C.c_int, _vp, _vp,
                                 C.POINTER(_Forcing), _vp, C.c_int, _vp]
    L.nf_field_advance.argtypes = [_vp, C.POINTER(_Model), C.c_int, _vp, _vp, C.c_int, C.c_double, C.c_int, _vp,
                                   _vp, _vp]
    L.nf_adjoint.argtypes = [_vp, _vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, _vp, _vp,
                             C.POINTER(_Forcing), _vp, _vp, _vp, _vp]
    _lib = L
    return L


def _check(st: int):
    if st != 0:
        raise NFError(st, lib().nf_last_error().decode(errors="replace"))


def _stream(t: torch.Tensor | None = None):
    dev = t.device if t is not None else None
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _dptr(t: torch.Tensor, dtype: torch.dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _kernel(kp) -> _Kernel:
    """(A1, s1, A2, s2) or (A1, s1, A2, s2, period); period L > 0: doubly periodic distance
    on the square of side L (x and y differences to their nearest images)."""
    v = [float(x) for x in kp]
    if len(v) == 4:
        v.append(0.0)
    if len(v) != 5:
        raise ValueError("kernel must be (A1, s1, A2, s2[, period])")
    return _Kernel(*v)


# ------------------------------------------------------------------------ §3.1-3.3

def nf_build_stencils(nodes: torch.Tensor, tris: torch.Tensor, k: int) -> torch.Tensor:
    """k nearest nodes (ascending (d^2, index)) to each element centroid.
    nodes: n x dim float64 CUDA, tris: m x 3 int32 CUDA -> m x k int32."""
    n, dim = nodes.shape
    m = tris.shape[0]
    out = torch.empty((m, k), dtype=torch.int32, device=nodes.device)
    _check(lib().nf_build_stencils(_dptr(nodes, torch.float64, "nodes"), n, dim, _dptr(tris, torch.int32, "tris"),
                                   m, int(k), _dptr(out, torch.int32, "stencils"), _stream(nodes)))
    return out


def nf_build_stencils_at(nodes: torch.Tensor, centers: torch.Tensor, k: int) -> torch.Tensor:
    """k nearest nodes (ascending (d^2, index)) to each given centre.
    nodes: n x dim float64 CUDA, centers: m x dim float64 CUDA -> m x k int32."""
    n, dim = nodes.shape
    m = centers.shape[0]
    if centers.dim() != 2 or centers.shape[1] != dim:
        raise ValueError(f"centers must be m x {dim}")
    out = torch.empty((m, k), dtype=torch.int32, device=nodes.device)
    _check(lib().nf_build_stencils_at(_dptr(nodes, torch.float64, "nodes"), n, dim,
                                      _dptr(centers, torch.float64, "centers"), m, int(k),
                                      _dptr(out, torch.int32, "stencils"), _stream(nodes)))
    return out


def nf_quad_weights_opts(nodes: torch.Tensor, tris: torch.Tensor, stencils: torch.Tensor, opts: dict,
                         normals: torch.Tensor | None = None) -> torch.Tensor:
    """nf_quad_weights with an options struct: opts = {dim, phs_order, poly_deg, curved}."""
    n = nodes.shape[0]
    m, k = stencils.shape
    o = _QuadOpts(int(opts["dim"]), int(opts.get("phs_order", 3)), int(opts["poly_deg"]), int(opts["curved"]))
    q = torch.empty(n, dtype=torch.float64, device=nodes.device)
    bad = C.c_int64(-1)
    nptr = _dptr(normals, torch.float64, "normals") if normals is not None else None
    _check(lib().nf_quad_weights_opts(_dptr(nodes, torch.float64, "nodes"), nptr, n, _dptr(tris, torch.int32, "tris"),
                                      m, _dptr(stencils, torch.int32, "stencils"), k, C.byref(o),
                                      _dptr(q, torch.float64, "q"), C.byref(bad), _stream(nodes)))
    return q


def nf_quad_weights(nodes: torch.Tensor, tris: torch.Tensor, stencils: torch.Tensor, deg: int,
                    normals: torch.Tensor | None = None) -> torch.Tensor:
    """RBF-QF node weights (float64, n)."""
    n, dim = nodes.shape
    m, k = stencils.shape
    q = torch.empty(n, dtype=torch.float64, device=nodes.device)
    bad = C.c_int64(-1)
    nptr = _dptr(normals, torch.float64, "normals") if normals is not None else None
    _check(lib().nf_quad_weights(_dptr(nodes, torch.float64, "nodes"), nptr, n, dim, _dptr(tris, torch.int32, "tris"),
                                 m, _dptr(stencils, torch.int32, "stencils"), k, int(deg),
                                 _dptr(q, torch.float64, "q"), C.byref(bad), _stream(nodes)))
    return q


# ------------------------------------------------------------------------ operator

class Forcing:
    """Forcing descriptor: kind 0 (none), 1 (manufactured, two eigenfunctions) or 2 (the
    moving-Gaussian manufactured solution on the periodic square: c, radius, sigma, scale)."""

    def __init__(self, kind=0, Y1=None, Y2=None, c=0.0, a0=0.0, lam=(0.0, 0.0, 0.0), radius=0.0, sigma=0.0,
                 scale=1.0):
        self.kind, self.Y1, self.Y2, self.c, self.a0, self.lam = kind, Y1, Y2, c, a0, tuple(lam)
        self.radius, self.sigma, self.scale = radius, sigma, scale

    @classmethod
    def flat(cls, c=0.1, radius=0.2, sigma=1.1, scale=1.0):
        return cls(FORCE_MMS_FLAT, c=c, radius=radius, sigma=sigma, scale=scale)

    @classmethod
    def sphere(cls, c=0.5, a0=0.3):
        """The manufactured solution on the unit sphere, with Y1 = z/2, Y2 = x y and the
        eigenvalues taken by the library from the operator."""
        return cls(FORCE_MMS_SPHERE, c=c, a0=a0)

    def _struct(self):
        y1 = _dptr(self.Y1, torch.float32, "Y1").value if self.Y1 is not None else None
        y2 = _dptr(self.Y2, torch.float32, "Y2").value if self.Y2 is not None else None
        return _Forcing(int(self.kind), y1, y2, float(self.c), float(self.a0), *(float(v) for v in self.lam),
                        float(self.radius), float(self.sigma), float(self.scale))


class Operator:
    """Owning handle for ``nf_operator`` (W diag(q) on n nodes, one of three paths)."""

    def __init__(self, x: torch.Tensor, q: torch.Tensor, kernel, path: int = MATRIX_FREE):
        self.n = int(x.shape[0])
        self.kernel = tuple(float(v) for v in kernel)
        self.path = int(path)
        self.device = x.device
        h = C.c_void_p()
        _check(lib().nf_operator_create(_dptr(x, torch.float32, "x"), _dptr(q, torch.float32, "q"), self.n,
                                        _kernel(kernel), self.path, _stream(x), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("operator destroyed")
        return self._h

    def profile(self, enable=True, ring: int = 1):
        """Record events around each stage's nonlocal kernels in captured RK4 steps; the
        last ``ring`` steps keep their own timings (read with :meth:`kernel_ms_history`)."""
        _check(lib().nf_operator_profile(self.handle, max(1, int(ring)) if enable else 0))

    def kernel_ms(self):
        """Durations (ms) of the four stages' nonlocal kernels in the last RK4 step."""
        out = (C.c_float * 4)()
        _check(lib().nf_operator_kernel_ms(self.handle, out))
        return list(out)

    def kernel_ms_history(self, steps: int):
        """Stage durations (ms) of the last ``steps`` profiled RK4 steps, oldest first
        (a list of 4-element lists)."""
        out = (C.c_float * (4 * int(steps)))()
        _check(lib().nf_operator_kernel_ms_history(self.handle, int(steps), out))
        v = list(out)
        return [v[4 * k:4 * k + 4] for k in range(int(steps))]

    def launch_shape(self):
        """(rows per warp, tile columns, column splits) of the matrix-free pair kernel."""
        r, t, s = C.c_int(), C.c_int(), C.c_int()
        _check(lib().nf_operator_launch_shape(self.handle, C.byref(r), C.byref(t), C.byref(s)))
        return {"rows_per_warp": r.value, "tile_cols": t.value, "splits": s.value}

    def mf_schedule(self, schedule: int):
        """Single-trajectory matrix-free schedule: MF_AUTO, MF_SYMMETRIC, MF_PACKED, or the
        symmetric kernel with a fixed node block (MF_SYMMETRIC_512 / MF_SYMMETRIC_1024)."""
        _check(lib().nf_operator_mf_schedule(self.handle, int(schedule)))
        return self

    def mf_cull(self, enable: bool = True):
        """Skip block pairs whose every pair contributes exactly zero in FP32 (bit-identical
        results); returns (live block pairs, total block pairs)."""
        live, tot = C.c_int64(), C.c_int64()
        _check(lib().nf_operator_mf_cull(self.handle, int(enable), C.byref(live), C.byref(tot), _stream()))
        return live.value, tot.value

    def check(self):
        _check(lib().nf_operator_check(self.handle, _stream()))

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            torch.cuda.synchronize(self.device)
            lib().nf_operator_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GroupedOperator(Operator):
    """Owning handle for a grouped operator (``nf_operator_group``): several
    DENSE_BF16X2 operators advanced together by the tcgen05 tensor-core GEMM.  States
    are the concatenation over members of their B_g x n_g blocks; the members must stay
    alive while the group is used."""

    def __init__(self, members, B_per_op):
        self.members = list(members)
        self.B_per_op = [int(b) for b in B_per_op]
        self.n = sum(m.n * b for m, b in zip(self.members, self.B_per_op))
        self.B = sum(self.B_per_op)
        self.path = 3
        self.device = self.members[0].device
        self.kernel = self.members[0].kernel
        arr = (C.c_void_p * len(self.members))(*[m.handle.value for m in self.members])
        bs = (C.c_int * len(self.members))(*self.B_per_op)
        h = C.c_void_p()
        _check(lib().nf_operator_group(arr, bs, len(self.members), _stream(), C.byref(h)))
        self._h = h

    def tuning(self):
        """The launch configuration the autotuner chose at creation."""
        d, sp, c, g, ms = C.c_int(), C.c_int(), C.c_double(), C.c_int(), C.c_float()
        _check(lib().nf_operator_group_tuning(self.handle, C.byref(d), C.byref(sp), C.byref(c), C.byref(g),
                                              C.byref(ms)))
        return {"ring_depth": d.value, "traj_split": sp.value, "lpt_coef": c.value, "subgroups": g.value,
                "ms_per_launch": ms.value}

    def configure(self, ring_depth: int, traj_split: int, lpt_coef: float):
        """Set the launch configuration instead of the autotuner's choice."""
        _check(lib().nf_operator_group_configure(self.handle, int(ring_depth), int(traj_split), float(lpt_coef),
                                                 _stream()))
        return self

    def split(self, flat: torch.Tensor):
        """View a concatenated state as the list of per-member (B_g x n_g) blocks."""
        out, off = [], 0
        for m, b in zip(self.members, self.B_per_op):
            out.append(flat[off:off + b * m.n].view(b, m.n))
            off += b * m.n
        return out


def _per_traj(v, B, device):
    if isinstance(v, torch.Tensor):
        return v.to(device=device, dtype=torch.float32).contiguous().expand(B).contiguous()
    return torch.full((B,), float(v), dtype=torch.float32, device=device)


def nf_nonlocal_apply(op: Operator, u: torch.Tensor, beta, theta, out: torch.Tensor | None = None) -> torch.Tensor:
    """I[b, i] = sum_j w(|x_i - x_j|) q_j f_b(u[b, j]); u: B x n float32 CUDA (for a
    grouped operator: the flat concatenation of the members' B_g x n_g blocks)."""
    if isinstance(op, GroupedOperator):
        u2, B = u.reshape(-1), op.B
    else:
        u2 = u if u.dim() == 2 else u.view(1, -1)
        B = u2.shape[0]
    be, th = _per_traj(beta, B, u.device), _per_traj(theta, B, u.device)
    I = out if out is not None else torch.empty_like(u2)
    _check(lib().nf_nonlocal_apply(op.handle, _dptr(u2, torch.float32, "u"), B, _dptr(be, torch.float32, "beta"),
                                   _dptr(th, torch.float32, "theta"), _dptr(I, torch.float32, "I"), _stream(u)))
    return I if u.dim() == 2 else I.view(-1)


def nf_nonlocal_apply_noalloc(x: torch.Tensor, q: torch.Tensor, u: torch.Tensor, kernel, beta: float, theta: float,
                              out: torch.Tensor) -> torch.Tensor:
    """Single-trajectory nonlocal sum that allocates nothing (neither here nor in the
    library): for callers that cannot allocate device memory at call time.  ``out``
    must be preallocated (n float32).  n <= 32768; calls that overlap on the GPU race.
    x must be n x 3 and q, u, out hold n elements each, all on the current CUDA device
    (checked here: the library trusts the sizes it is given)."""
    n = int(x.shape[0]) if x.dim() >= 1 else 0
    if x.dim() != 2 or tuple(x.shape) != (n, 3):
        raise ValueError(f"x must be n x 3, got {tuple(x.shape)}")
    for name, t in (("q", q), ("u", u), ("out", out)):
        if t.numel() != n:
            raise ValueError(f"{name} must hold n = {n} elements, got {t.numel()}")
    cur = torch.cuda.current_device()
    for name, t in (("x", x), ("q", q), ("u", u), ("out", out)):
        if not t.is_cuda or t.device.index != cur:
            raise ValueError(f"{name} must be on the current CUDA device cuda:{cur}, got {t.device}")
    _check(lib().nf_nonlocal_apply_noalloc(_dptr(x, torch.float32, "x"), _dptr(q, torch.float32, "q"), n,
                                           _kernel(kernel), _dptr(u, torch.float32, "u"), float(beta), float(theta),
                                           _dptr(out, torch.float32, "I"), _stream(x)))
    return out


def nf_noalloc_status():
    """Synchronise the current stream and raise NFError (NF_ERR_TIMEOUT) if the last
    allocation-free sum on this device gave up a bounded wait (its output is then NaN)."""
    _check(lib().nf_noalloc_status(_stream()))


def nf_noalloc_limits(n: int):
    """(largest n accepted, column splits the scratch holds, splits a call on n nodes uses)."""
    mx, ms, sp = C.c_int64(), C.c_int(), C.c_int()
    _check(lib().nf_noalloc_limits(int(n), C.byref(mx), C.byref(ms), C.byref(sp)))
    return mx.value, ms.value, sp.value


def nf_selftest_noalloc_flag(out: torch.Tensor):
    """Record a timeout in the allocation-free call's flag and run its final reduction into
    ``out`` (n float32): every entry becomes NaN.  Exercises the failure path without a wait."""
    _check(lib().nf_selftest_noalloc_flag(out.numel(), _dptr(out, torch.float32, "I"), _stream(out)))
    return out


PROBE_FMA, PROBE_FMA2, PROBE_EX2, PROBE_FMA2_OUTER = 0, 1, 2, 3


def nf_probe_pipe(kind: int, iters: int = 20000):
    """Measured rate of one instruction kind on every SM (PROBE_FMA: fma.rn.f32 lane
    operations, PROBE_FMA2: fma.rn.f32x2 lane operations, PROBE_EX2: SFU ex2,
    PROBE_FMA2_OUTER: fma.rn.f32x2 as an outer product with distinct operands): returns
    (operations per clock per SM, SM MHz during the probe, wall ms)."""
    r, mhz, ms = C.c_double(), C.c_double(), C.c_float()
    _check(lib().nf_probe_pipe(int(kind), int(iters), C.byref(r), C.byref(mhz), C.byref(ms), _stream()))
    return r.value, mhz.value, ms.value


def nf_rk4_advance(op: Operator, u: torch.Tensor, t0: float, dt: float, nsteps: int, beta, theta,
                   forcing: Forcing | None = None, ckpt: torch.Tensor | None = None, C_every: int = 1):
    """Advance u (B x n float32 CUDA, in place) by nsteps RK4 steps (grouped operator:
    u is the flat concatenation of the members' B_g x n_g blocks)."""
    if isinstance(op, GroupedOperator):
        u2, B = u.reshape(-1), op.B
    else:
        u2 = u if u.dim() == 2 else u.view(1, -1)
        B = u2.shape[0]
    be, th = _per_traj(beta, B, u.device), _per_traj(theta, B, u.device)
    f = C.byref(forcing._struct()) if forcing is not None else None
    cp = _dptr(ckpt, torch.float32, "ckpt") if ckpt is not None else None
    _check(lib().nf_rk4_advance(op.handle, _dptr(u2, torch.float32, "u"), B, float(t0), float(dt), int(nsteps),
                                _dptr(be, torch.float32, "beta"), _dptr(th, torch.float32, "theta"), f, cp,
                                int(C_every), _stream(u)))
    # keep the per-trajectory arrays alive until the queued work has consumed them
    op._keep = (be, th, forcing)
    return u


MODEL_FIELD, MODEL_DEPRESSION = 0, 1
RATE_SIGMOID, RATE_SMOOTHSTEP = 0, 1


def nf_field_advance(op: Operator, u: torch.Tensor, dt: float, nsteps: int, beta=1.0, theta=0.0,
                     s: torch.Tensor | None = None, rate: int = RATE_SIGMOID, a: float = 0.06, b: float = 0.54,
                     tau: float = 1.0, beta_d: float = 0.0, integrator: str = "rk4"):
    """Advance a §5 model in place: the neural field (s None) or the synaptic-depression
    model (s: B x n efficacy), sigmoid or C^4 smooth-step rate, RK4 or AB5."""
    u2 = u if u.dim() == 2 else u.view(1, -1)
    B = u2.shape[0]
    s2 = None if s is None else (s if s.dim() == 2 else s.view(1, -1))
    be, th = _per_traj(beta, B, u.device), _per_traj(theta, B, u.device)
    m = _Model(MODEL_DEPRESSION if s is not None else MODEL_FIELD, int(rate), float(a), float(b), float(tau),
               float(beta_d))
    integ = {"rk4": 0, "ab5": 1}[integrator]
    _check(lib().nf_field_advance(op.handle, C.byref(m), integ, _dptr(u2, torch.float32, "u"),
                                  _dptr(s2, torch.float32, "s") if s2 is not None else None, B, float(dt),
                                  int(nsteps), _dptr(be, torch.float32, "beta"), _dptr(th, torch.float32, "theta"),
                                  _stream(u)))
    op._keep = (be, th)
    return (u, s) if s is not None else u


def nf_adjoint(op: Operator, ckpt: torch.Tensor, C_every: int, t0: float, dt: float, nsteps: int, beta, theta,
               lambda_T: torch.Tensor, forcing: Forcing | None = None):
    """Discrete RK4 adjoint: returns (dL/du0 (B x n), dL/d(A1,s1,A2,s2) (B x 4))."""
    lam = lambda_T if lambda_T.dim() == 2 else lambda_T.view(1, -1)
    B, n = lam.shape
    be, th = _per_traj(beta, B, lam.device), _per_traj(theta, B, lam.device)
    gu = torch.empty_like(lam)
    gk = torch.empty((B, 4), dtype=torch.float32, device=lam.device)
    f = C.byref(forcing._struct()) if forcing is not None else None
    _check(lib().nf_adjoint(op.handle, _dptr(ckpt, torch.float32, "ckpt"), int(C_every), B, float(t0), float(dt),
                            int(nsteps), _dptr(be, torch.float32, "beta"), _dptr(th, torch.float32, "theta"), f,
                            _dptr(lam, torch.float32, "lambda_T"), _dptr(gu, torch.float32, "grad_u0"),
                            _dptr(gk, torch.float32, "grad_kernel"), _stream(lam)))
    op._keep = (be, th, forcing)
    return gu, gk


class NeuralFieldRK4(torch.autograd.Function):
    """u(T) after ``nsteps`` classical RK4 steps of Eq. (2.9) from ``u0``, differentiable in u0
    and in the kernel parameters (A1, s1, A2, s2).

    ``NeuralFieldRK4.apply(u0, kernel_params, x, q, beta, theta, t0, dt, nsteps[, C_every[,
    forcing[, period]]])`` (positional; defaults 10, None, 0.0): forward builds a matrix-free operator from the values of
    ``kernel_params`` (a 4-element tensor) and runs :func:`nf_rk4_advance` with a checkpoint
    every ``C_every`` steps; backward runs :func:`nf_adjoint` from the incoming gradient of
    u(T) and returns dL/du0 and dL/d(kernel_params) (summed over trajectories).  u0: n or
    B x n float32 CUDA; x: n x 3, q: n float32 CUDA (constants)."""

    @staticmethod
    def forward(ctx, u0, kernel_params, x, q, beta, theta, t0, dt, nsteps, C_every=10, forcing=None, period=0.0):
        kp = [float(v) for v in kernel_params.detach().reshape(-1).cpu().tolist()]
        if len(kp) != 4:
            raise ValueError("kernel_params must hold (A1, s1, A2, s2)")
        op = Operator(x, q, kp + [float(period)], MATRIX_FREE)
        squeeze = u0.dim() == 1
        u = u0.detach().to(torch.float32).reshape(1 if squeeze else u0.shape[0], -1).contiguous().clone()
        B, n = u.shape
        C_every = max(1, int(C_every))
        ck = torch.empty((int(nsteps) // C_every + 1, B, n), dtype=torch.float32, device=u.device)
        nf_rk4_advance(op, u, t0, dt, int(nsteps), beta, theta, forcing=forcing, ckpt=ck, C_every=C_every)
        ctx.save_for_backward(ck)
        ctx.op = op
        ctx.args = (C_every, float(t0), float(dt), int(nsteps), beta, theta, forcing, squeeze, kernel_params)
        return u.view(-1) if squeeze else u

    @staticmethod
    def backward(ctx, grad_out):
        (ck,) = ctx.saved_tensors
        C_every, t0, dt, nsteps, beta, theta, forcing, squeeze, kparams = ctx.args
        lam = grad_out.detach().to(torch.float32).reshape(ck.shape[1], ck.shape[2]).contiguous()
        gu, gk = nf_adjoint(ctx.op, ck, C_every, t0, dt, nsteps, beta, theta, lam, forcing=forcing)
        g_kernel = gk.sum(0).to(dtype=kparams.dtype, device=kparams.device).reshape(kparams.shape)
        g_u0 = gu.view(-1) if squeeze else gu
        return (g_u0, g_kernel) + (None,) * 10


def nf_mms_sphere_eigs(kernel):
    lam = (C.c_double * 3)()
    _check(lib().nf_mms_sphere_eigs(_kernel(kernel), lam))
    return tuple(lam)
