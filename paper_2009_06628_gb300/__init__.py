"""Thin Python binding of libchns (the C-ABI declared in include/chns.h).

Only argument marshalling happens here: torch tensors supply device memory and the
current CUDA stream; every step of the hot path runs in the library's CUDA kernels.
The binding refuses to work without the compiled library (there is no CPU path).
"""
import ctypes
import os

import numpy as np
import torch

__all__ = ["lib", "load", "Params", "SolverOpts", "Stats", "ChnsError", "Mesh", "residual", "jvp", "vjp",
           "newton_step", "mass", "energy", "initial_mu", "kernel_launches", "step_adjoint", "free_energy_grad",
           "mu_rhs_vjp", "mass_solve", "LIB_PATH"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libchns.so")

STATUS = {0: "CHNS_OK", 1: "CHNS_EINVAL", 2: "CHNS_ENOTSORTED", 3: "CHNS_ENOTCOMPLETE", 4: "CHNS_ENOTBALANCED",
          5: "CHNS_ENOMEM", 6: "CHNS_ECUDA", 7: "CHNS_ENAN", 8: "CHNS_ENOCONV", 9: "CHNS_EBREAKDOWN",
          10: "CHNS_ETAU"}


class ChnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("pin_pressure", ctypes.c_int32), ("Re", ctypes.c_double),
                ("We", ctypes.c_double), ("Pe", ctypes.c_double), ("Cn", ctypes.c_double), ("Fr", ctypes.c_double),
                ("rho_ratio", ctypes.c_double), ("eta_ratio", ctypes.c_double), ("dt", ctypes.c_double),
                ("C_I", ctypes.c_double), ("C_phi", ctypes.c_double)]

    @classmethod
    def make(cls, dim, Re, We, Pe, Cn, Fr, rho_ratio, eta_ratio, dt, C_I=6.0, C_phi=6.0, pin_pressure=2,
             **_ignored):
        return cls(dim=dim, pin_pressure=pin_pressure, Re=Re, We=We, Pe=Pe, Cn=Cn, Fr=Fr, rho_ratio=rho_ratio,
                   eta_ratio=eta_ratio, dt=dt, C_I=C_I, C_phi=C_phi)


class SolverOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("krylov_rtol", ctypes.c_double),
                ("max_newton", ctypes.c_int32), ("max_krylov", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("pc_type", ctypes.c_int32), ("pc_degree", ctypes.c_int32),
                ("ew_eta0", ctypes.c_double), ("guess", ctypes.c_int32)]

    @classmethod
    def make(cls, rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, max_newton=20, max_krylov=2000, restart=60,
             precision=1, pc_type=1, pc_degree=8, ew_eta0=0.0, guess=0):
        return cls(rtol=rtol, atol=atol, krylov_rtol=krylov_rtol, max_newton=max_newton, max_krylov=max_krylov,
                   restart=restart, precision=precision, pc_type=pc_type, pc_degree=pc_degree, ew_eta0=ew_eta0,
                   guess=guess)


class Stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int32), ("krylov_its", ctypes.c_int32), ("jvp_calls", ctypes.c_int32),
                ("reason", ctypes.c_int32), ("res0", ctypes.c_double), ("res_final", ctypes.c_double),
                ("du_norm", ctypes.c_double), ("jvp_ms", ctypes.c_double), ("pc_ms", ctypes.c_double),
                ("apply_ms", ctypes.c_double), ("orth_ms", ctypes.c_double),
                ("res_hist", ctypes.c_double * 32), ("krylov_hist", ctypes.c_int32 * 32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.endswith("_hist")}
        d["res_hist"] = list(self.res_hist[:min(self.newton_its + 1, 32)])
        d["krylov_hist"] = list(self.krylov_hist[:min(self.newton_its, 32)])
        return d


_lib = None

# (name, restype, argtypes) of every entry point in include/chns.h
P = ctypes.c_void_p
SIGNATURES = [
    ("chns_mesh_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    ("chns_mesh_destroy", None, [P]),
    ("chns_mesh_create_q2", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    ("chns_mesh_order", ctypes.c_int32, [P]),
    ("chns_mesh_num_nodes", ctypes.c_int64, [P]),
    ("chns_mesh_num_elements", ctypes.c_int64, [P]),
    ("chns_mesh_num_hanging", ctypes.c_int64, [P]),
    ("chns_mesh_dim", ctypes.c_int32, [P]),
    ("chns_mesh_node_coords", ctypes.c_int, [P, P]),
    ("chns_mesh_set_velocity_bc", ctypes.c_int, [P, P, P]),
    ("chns_mesh_set_scatter", ctypes.c_int, [P, ctypes.c_int32]),
    ("chns_mesh_num_colours", ctypes.c_int32, [P]),
    ("chns_residual", ctypes.c_int, [P, P, P, P, P, P]),
    ("chns_jvp", ctypes.c_int, [P, P, P, P, P, P, ctypes.c_int32, P]),
    ("chns_vjp", ctypes.c_int, [P, P, P, P, P, P, P, P, P]),
    ("chns_newton_step", ctypes.c_int, [P, P, P, P, P, P, P]),
    ("chns_mass", ctypes.c_int, [P, P, P, P]),
    ("chns_energy", ctypes.c_int, [P, P, P, P, P]),
    ("chns_initial_mu", ctypes.c_int, [P, P, P, P]),
    ("chns_mass_static", ctypes.c_int, [P, P, P, P]),
    ("chns_step_adjoint", ctypes.c_int, [P, P, P, P, P, P, P, P, P, P, P]),
    ("chns_free_energy_grad", ctypes.c_int, [P, P, P, P, P, P]),
    ("chns_mu_rhs_vjp", ctypes.c_int, [P, P, P, P, P, P, P]),
    ("chns_mass_solve", ctypes.c_int, [P, P, P, P]),
    ("chns_transfer_create", ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_void_p)]),
    ("chns_transfer_destroy", None, [P]),
    ("chns_transfer_nnz", ctypes.c_int64, [P]),
    ("chns_transfer_apply", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P, P, P]),
    ("chns_coarsen_leaves", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P, ctypes.c_int32, P, P,
                                           ctypes.POINTER(ctypes.c_int64)]),
    ("chns_adapt_flags", ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, P, P]),
    ("chns_adapt_leaves", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P, P, ctypes.c_int32,
                                         ctypes.c_int32, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int32)]),
    ("chns_fma_peak", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int64, P, P]),
    ("chns_kernel_launches", ctypes.c_int64, []),
    ("chns_last_error", ctypes.c_char_p, []),
]


def load(path=None):
    """Load libchns.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libchns.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def lib():
    return load()


def _check(code):
    if code != 0:
        raise ChnsError(code, load().chns_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=torch.float64):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """Owns a chns_mesh built from an (n, 4) int32 leaf array (x, y, z, level)."""

    def __init__(self, dim, max_level, leaves, lo=0.0, hi=1.0):
        L = load()
        leaves = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32))
        if leaves.ndim != 2 or leaves.shape[1] != 4:
            raise ValueError("leaves must be an (n, 4) int32 array")
        h = ctypes.c_void_p()
        _check(L.chns_mesh_create(int(dim), int(max_level), int(leaves.shape[0]),
                                  leaves.ctypes.data_as(ctypes.c_void_p), float(lo), float(hi), ctypes.byref(h)))
        self._h = h
        self.leaves = leaves
        self.dim = int(dim)
        self.nf = self.dim + 3
        self.max_level = int(max_level)
        self.lo, self.hi = float(lo), float(hi)
        self.N = int(L.chns_mesh_num_nodes(h))
        self.E = int(L.chns_mesh_num_elements(h))
        self.H = int(L.chns_mesh_num_hanging(h))

    @property
    def handle(self):
        return self._h

    def node_coords(self):
        out = np.zeros((self.N, self.dim), dtype=np.int32)
        _check(load().chns_mesh_node_coords(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_velocity_bc(self, face_mask, values=None):
        """face_mask: 2 * dim ints (face 2k: x_k = lo, 2k + 1: x_k = hi; bit c = component c
        Dirichlet); values: optional (N, dim) FP64 CUDA tensor of prescribed velocities."""
        fm = np.ascontiguousarray(np.asarray(face_mask, dtype=np.uint8))
        if fm.shape != (2 * self.dim,):
            raise ValueError("face_mask needs 2 * dim entries")
        vp = _ptr(values.contiguous()) if values is not None else None
        _check(load().chns_mesh_set_velocity_bc(self._h, fm.ctypes.data_as(ctypes.c_void_p), vp))

    def set_scatter(self, mode):
        """0 atomics, 1 element colouring (deterministic), 2 warp-aggregated atomics."""
        _check(load().chns_mesh_set_scatter(self._h, int(mode)))

    @property
    def num_colours(self):
        return int(load().chns_mesh_num_colours(self._h))

    def node_x(self):
        return self.lo + (self.hi - self.lo) * self.node_coords().astype(np.float64) / float(1 << self.max_level)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().chns_mesh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def residual(mesh, prm, U_old, U_new, out=None):
    out = torch.empty_like(U_new) if out is None else out
    _check(load().chns_residual(mesh.handle, ctypes.byref(prm), _ptr(U_old), _ptr(U_new), _ptr(out), _stream()))
    return out


def jvp(mesh, prm, U_old, U_lin, x, out=None):
    """y = J(U_lin) x in the dtype of the inputs (float64 or float32)."""
    dt = x.dtype
    prec = {torch.float64: 0, torch.float32: 1}[dt]
    out = torch.empty_like(x) if out is None else out
    _check(load().chns_jvp(mesh.handle, ctypes.byref(prm), _ptr(U_old, dt), _ptr(U_lin, dt), _ptr(x, dt),
                           _ptr(out, dt), prec, _stream()))
    return out


def vjp(mesh, prm, U_old, U_lin, w, want_old=True, want_cn=True):
    gn = torch.empty_like(w)
    go = torch.empty_like(w) if want_old else None
    gc = torch.empty(1, dtype=torch.float64, device=w.device) if want_cn else None
    _check(load().chns_vjp(mesh.handle, ctypes.byref(prm), _ptr(U_old), _ptr(U_lin), _ptr(w), _ptr(gn),
                           _ptr(go) if go is not None else None, _ptr(gc) if gc is not None else None, _stream()))
    return gn, go, gc


def newton_step(mesh, prm, opts, U_old, U_out=None, check=True):
    """One implicit step from U_old; with opts.guess = 1, U_out (required) holds the first
    Newton iterate on entry."""
    if opts.guess and U_out is None:
        raise ValueError("opts.guess = 1 needs U_out holding the first iterate")
    U_out = torch.empty_like(U_old) if U_out is None else U_out
    st = Stats()
    code = load().chns_newton_step(mesh.handle, ctypes.byref(prm), ctypes.byref(opts), _ptr(U_old), _ptr(U_out),
                                   ctypes.byref(st), _stream())
    if check:
        _check(code)
    return U_out, st


def mass(mesh, U):
    out = ctypes.c_double()
    _check(load().chns_mass(mesh.handle, _ptr(U), ctypes.byref(out), _stream()))
    return out.value


def energy(mesh, prm, U):
    out = (ctypes.c_double * 3)()
    _check(load().chns_energy(mesh.handle, ctypes.byref(prm), _ptr(U), out, _stream()))
    return tuple(out)


def step_adjoint(mesh, prm, opts, U_old, U_new, g, want_cn=True):
    """Cotangents (lambda, gU_old, gCn) of one implicit step for the cotangent g of U_new."""
    lam = torch.empty_like(g)
    go = torch.empty_like(g)
    gc = torch.zeros(1, dtype=torch.float64, device=g.device) if want_cn else None
    st = Stats()
    _check(load().chns_step_adjoint(mesh.handle, ctypes.byref(prm), ctypes.byref(opts), _ptr(U_old), _ptr(U_new),
                                    _ptr(g), _ptr(lam), _ptr(go), _ptr(gc) if gc is not None else None,
                                    ctypes.byref(st), _stream()))
    return lam, go, gc, st


def free_energy_grad(mesh, prm, U):
    """(dF/dU, dF/dCn) of the free-energy part F of E_tot."""
    g = torch.empty_like(U)
    d = ctypes.c_double()
    _check(load().chns_free_energy_grad(mesh.handle, ctypes.byref(prm), _ptr(U), _ptr(g), ctypes.byref(d),
                                        _stream()))
    return g, d.value


def mu_rhs_vjp(mesh, prm, U, lam):
    """((db/dphi)^T lam, lam^T db/dCn) of the potential right-hand side b(phi; Cn)."""
    g = torch.empty(U.shape[0], dtype=torch.float64, device=U.device)
    d = ctypes.c_double()
    _check(load().chns_mu_rhs_vjp(mesh.handle, ctypes.byref(prm), _ptr(U), _ptr(lam.contiguous()), _ptr(g),
                                  ctypes.byref(d), _stream()))
    return g, d.value


def mass_solve(mesh, rhs):
    x = torch.empty_like(rhs)
    _check(load().chns_mass_solve(mesh.handle, _ptr(rhs.contiguous()), _ptr(x), _stream()))
    return x


def kernel_launches():
    """Kernels launched by libchns so far in this process."""
    return int(load().chns_kernel_launches())


def initial_mu(mesh, prm, U):
    """Overwrite the mu field of U (in place) with the discrete mu^0 of its phi."""
    _check(load().chns_initial_mu(mesh.handle, ctypes.byref(prm), _ptr(U), _stream()))
    return U


def fma_peak(precision=1, iters=20000):
    """Measured CUDA-core FMA throughput of the current GPU in flop/s (precision 1: FP32,
    0: FP64), timed with CUDA events on the current stream."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    scratch = torch.empty(4 * sms * 256, dtype=torch.float64, device="cuda")
    out = ctypes.c_double(0.0)
    _check(load().chns_fma_peak(precision, iters, ctypes.c_void_p(scratch.data_ptr()), scratch.numel() * 8,
                                ctypes.byref(out), _stream()))
    return out.value


class Transfer:
    """Owns a chns_transfer: Q1 interpolation from mesh `src` to the nodes of mesh `dst`."""

    def __init__(self, src, dst):
        h = ctypes.c_void_p()
        _check(load().chns_transfer_create(src.handle, dst.handle, ctypes.byref(h)))
        self._h = h
        self.n_src, self.n_dst = src.N, dst.N

    @property
    def nnz(self):
        return int(load().chns_transfer_nnz(self._h))

    def apply(self, u, transpose=False):
        """P u (u: n_src x nf) or P^T u (u: n_dst x nf), FP64 CUDA tensors."""
        u = u.contiguous()
        nf = 1 if u.dim() == 1 else u.shape[1]
        rows = self.n_src if transpose else self.n_dst
        out = torch.empty((rows,) + tuple(u.shape[1:]), dtype=torch.float64, device=u.device)
        _check(load().chns_transfer_apply(self._h, nf, 1 if transpose else 0, _ptr(u), _ptr(out), _stream()))
        return out

    def close(self):
        if self._h and self._h.value:
            load().chns_transfer_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def coarsen_leaves(dim, max_level, leaves, cap):
    """Host-only: (capped leaves (m, 4) int32 with anchors in units of 2^-cap, map (n,) int32)."""
    import numpy as np
    lv = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32).reshape(-1, 4))
    out = np.zeros_like(lv)
    fmap = np.zeros(lv.shape[0], dtype=np.int32)
    n = ctypes.c_int64(0)
    _check(load().chns_coarsen_leaves(dim, max_level, lv.shape[0], lv.ctypes.data_as(ctypes.c_void_p), cap,
                                      out.ctypes.data_as(ctypes.c_void_p), fmap.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(n)))
    return out[:n.value].copy(), fmap


def adapt_flags(mesh, U, phi_threshold, min_level, max_level):
    """Per-element int8 flags on the device: +1 refine, -1 coarsening candidate, 0 keep."""
    flags = torch.empty(mesh.E, dtype=torch.int8, device=U.device)
    _check(load().chns_adapt_flags(mesh.handle, _ptr(U), float(phi_threshold), int(min_level), int(max_level),
                                   ctypes.c_void_p(flags.data_ptr()), _stream()))
    return flags


def adapt_leaves(dim, max_level, leaves, flags, min_level, max_level_new):
    """Host-only: (new leaves (m, 4) int32, their max_level) after one adaptation pass."""
    lv = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32).reshape(-1, 4))
    fl = np.ascontiguousarray(np.asarray(flags, dtype=np.int8))
    if fl.shape[0] != lv.shape[0]:
        raise ValueError("one flag per leaf")
    cap = lv.shape[0] * (1 << dim) + 16
    while True:
        out = np.zeros((cap, 4), dtype=np.int32)
        n, L = ctypes.c_int64(0), ctypes.c_int32(0)
        code = load().chns_adapt_leaves(int(dim), int(max_level), lv.shape[0], lv.ctypes.data_as(ctypes.c_void_p),
                                        fl.ctypes.data_as(ctypes.c_void_p), int(min_level), int(max_level_new),
                                        out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n), ctypes.byref(L))
        if code != 0 and n.value > cap:
            cap = n.value
            continue
        _check(code)
        return out[:n.value].copy(), int(L.value)


def adapt(mesh, U, phi_threshold, min_level, max_level):
    """One remeshing pass: flags from U's phi on the GPU, the new leaf list on the host, the
    new mesh and U transferred to it by Q1 interpolation.  Returns (new mesh, new U, flags)."""
    fl = adapt_flags(mesh, U, phi_threshold, min_level, max_level).cpu().numpy()
    leaves, L = adapt_leaves(mesh.dim, mesh.max_level, mesh.leaves, fl, min_level, max_level)
    new = Mesh(mesh.dim, L, leaves, mesh.lo, mesh.hi)
    T = Transfer(mesh, new)
    return new, T.apply(U), fl


class MeshQ2(Mesh):
    """Owns a Q2 chns_mesh on the uniform octree of one level (node coordinates in units of
    2^-(level + 1))."""

    def __init__(self, dim, level, lo=0.0, hi=1.0):
        L = load()
        h = ctypes.c_void_p()
        _check(L.chns_mesh_create_q2(int(dim), int(level), float(lo), float(hi), ctypes.byref(h)))
        self._h = h
        self.leaves = None
        self.dim = int(dim)
        self.nf = self.dim + 3
        self.level = int(level)
        self.max_level = int(level) + 1       # resolution of the node coordinates
        self.lo, self.hi = float(lo), float(hi)
        self.N = int(L.chns_mesh_num_nodes(h))
        self.E = int(L.chns_mesh_num_elements(h))
        self.H = 0
