"""ctypes binding of librtcc.so (include/rtcc.h) with the same names.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Host arrays are numpy arrays; device arrays may be passed as torch
CUDA tensors (their data_ptr() is handed to the library).  Importing this
module raises if the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librtcc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_2205_05175_gb300.build")
_lib = C.CDLL(LIB_PATH)

P64, P32_TF32, P32_3XTF32, P32_BF16X3 = 0, 1, 2, 3
PRECISIONS = {"p64": P64, "tf32": P32_TF32, "3xtf32": P32_3XTF32, "bf16x3": P32_BF16X3}
RK4, CK, MIXED_RK4, GL2, GL2_NEWTON = 0, 1, 2, 3, 4
CARRIER_SIN, CARRIER_COS = 0, 1
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOCONV", 5: "DIVERGED",
          6: "STEP_UNDERFLOW", 7: "TIMEOUT", 8: "UNSUPPORTED"}


class rtcc_field_t(C.Structure):
    _fields_ = [("E0", C.c_double), ("omega", C.c_double), ("sigma", C.c_double), ("t0", C.c_double),
                ("pol", C.c_double * 3), ("carrier", C.c_int), ("sign", C.c_double)]


class rtcc_integrator_t(C.Structure):
    _fields_ = [("method", C.c_int), ("h", C.c_double), ("h1", C.c_double), ("h2", C.c_double),
                ("t_switch", C.c_double), ("tol", C.c_double), ("safety", C.c_double),
                ("h_min", C.c_double), ("h_max", C.c_double), ("max_rejects", C.c_int),
                ("nsteps", C.c_int), ("t_end", C.c_double), ("sweeps", C.c_int), ("krylov", C.c_int)]


class rtcc_profile_t(C.Structure):
    _fields_ = [("launches", C.c_longlong * 8), ("ms", C.c_double * 8), ("flops", C.c_double * 8),
                ("bytes", C.c_double * 8)]


KERNEL_CLASSES = ["tc_gemm", "f64_gemm", "pack", "unpack", "direct", "reduce", "add", "rk"]


class RtccError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


_vp, _dp, _ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
_sig = {
    "rtcc_create": [_vp, _vp, C.c_int, _vp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_vp)],
    "rtcc_create_frozen_core": [_vp, _vp, C.c_int, _vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_vp)],
    "rtcc_destroy": [_vp],
    "rtcc_state_size": [_vp, C.POINTER(C.c_size_t)],
    "rtcc_ground_state": [_vp, C.c_double, C.c_int, _dp, _dp],
    "rtcc_get_state": [_vp, C.c_int, _vp, _dp, _dp],
    "rtcc_set_state": [_vp, C.c_int, _vp, C.c_double, C.c_double],
    "rtcc_rhs": [_vp, _vp, C.POINTER(rtcc_field_t), _vp, _vp],
    "rtcc_rhs_vjp": [_vp, _vp, C.POINTER(rtcc_field_t), _vp, _vp, _vp],
    "rtcc_autotune": [_vp, _ip],
    "rtcc_dipole": [_vp, _vp],
    "rtcc_propagate": [_vp, C.POINTER(rtcc_field_t), C.POINTER(rtcc_integrator_t), C.c_int, _vp, _vp, _ip],
    "rtcc_last_stats": [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                        C.POINTER(C.c_longlong)],
    "rtcc_profile": [_vp, C.c_int, C.POINTER(rtcc_profile_t)],
    "rtcc_propagate_vjp": [_vp, C.POINTER(rtcc_field_t), C.c_double, C.c_int, _vp, C.c_int, _vp, _vp],
    "rtcc_spectrum": [_vp, _vp, C.c_int, C.POINTER(rtcc_field_t), C.c_double, C.c_double, C.c_double, _vp,
                      C.c_int, _vp],
    "rtcc_spectrum_pade": [_vp, _vp, C.c_int, C.POINTER(rtcc_field_t), C.c_double, C.c_double, _vp, C.c_int, _vp],
    "rtcc_selftest_gemm": [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp],
    "rtcc_selftest_timeout": [C.c_double],
    "rtcc_gemm_noalloc": [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp],
}
for _name, _args in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = C.c_int
_lib.rtcc_last_error.restype = C.c_char_p
_lib.rtcc_last_error.argtypes = []

EXPORTED = sorted(list(_sig) + ["rtcc_last_error"])


def rtcc_last_error() -> str:
    return _lib.rtcc_last_error().decode()


def _check(code):
    if code != 0:
        raise RtccError(code, rtcc_last_error())


def _ptr(x):
    """Pointer of a C-contiguous numpy array or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    raise TypeError(type(x))


def make_field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.0, 1.0), carrier=CARRIER_SIN, sign=1.0):
    f = rtcc_field_t()
    f.E0, f.omega, f.sigma, f.t0 = E0, omega, sigma, t0
    f.pol[0], f.pol[1], f.pol[2] = pol
    f.carrier, f.sign = carrier, sign
    return f


def make_integrator(method=RK4, h=0.05, h1=0.005, h2=0.05, t_switch=0.0, tol=1e-6, safety=0.84, h_min=1e-9,
                    h_max=1.0, max_rejects=50, nsteps=0, t_end=0.0, sweeps=0, krylov=0):
    i = rtcc_integrator_t()
    i.method, i.h, i.h1, i.h2, i.t_switch = method, h, h1, h2, t_switch
    i.tol, i.safety, i.h_min, i.h_max, i.max_rejects = tol, safety, h_min, h_max, max_rejects
    i.nsteps, i.t_end, i.sweeps, i.krylov = nsteps, t_end, sweeps, krylov
    return i


def _as_c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


class Handle:
    """Owner of one rtcc_handle_t (rtcc_create ... rtcc_destroy)."""

    def __init__(self, f, B, mu, o, v, ntraj=1, prec=P64, nfc=0):
        """nfc > 0 freezes the lowest nfc occupied orbitals (rtcc_create_frozen_core); the handle's
        state then covers the o - nfc active occupied orbitals."""
        f, B, mu = _as_c(f), _as_c(B), _as_c(mu)
        nmo = o + v
        assert f.shape == (nmo, nmo) and B.shape[1:] == (nmo, nmo) and mu.shape == (3, nmo, nmo)
        self.o, self.v, self.ntraj = o - nfc, v, ntraj
        h = C.c_void_p()
        if nfc:
            _check(_lib.rtcc_create_frozen_core(_ptr(f), _ptr(B), B.shape[0], _ptr(mu), o, v, nfc, ntraj, int(prec),
                                                C.byref(h)))
        else:
            _check(_lib.rtcc_create(_ptr(f), _ptr(B), B.shape[0], _ptr(mu), o, v, ntraj, int(prec), C.byref(h)))
        self.h = h
        n = C.c_size_t()
        _check(_lib.rtcc_state_size(self.h, C.byref(n)))
        self.ns = n.value

    def close(self):
        if getattr(self, "h", None):
            _lib.rtcc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def ground_state(self, tol=1e-10, maxiter=200):
        e = C.c_double()
        mu0 = (C.c_double * 3)()
        _check(_lib.rtcc_ground_state(self.h, tol, maxiter, C.byref(e), mu0))
        return e.value, np.array(mu0[:])

    def get_state(self, traj=0):
        y = np.zeros(self.ns, complex)
        t, hs = C.c_double(), C.c_double()
        _check(_lib.rtcc_get_state(self.h, traj, _ptr(y), C.byref(t), C.byref(hs)))
        return y, t.value, hs.value

    def set_state(self, traj, y, time=0.0, hstep=0.0):
        if isinstance(y, np.ndarray):
            y = np.ascontiguousarray(y, dtype=complex)
            assert y.size == self.ns
        _check(_lib.rtcc_set_state(self.h, traj, _ptr(y), time, hstep))

    def rhs(self, y, fields, times):
        """dy/dt for every trajectory: y (ntraj, ns) complex host array or torch tensor."""
        fa = (rtcc_field_t * self.ntraj)(*fields)
        tms = _as_c(times)
        if isinstance(y, np.ndarray):
            y = np.ascontiguousarray(y, dtype=complex)
            out = np.zeros_like(y)
        else:
            import torch
            out = torch.empty_like(y)
        _check(_lib.rtcc_rhs(self.h, _ptr(y), fa, _ptr(tms), _ptr(out)))
        return out

    def autotune(self):
        """Choose the tensor-core tiles of every batch size now; returns the GEMM shapes tuned."""
        n = C.c_int()
        _check(_lib.rtcc_autotune(self.h, C.byref(n)))
        return n.value

    def rhs_vjp(self, y, fields, times, u):
        """(d dydt / dy)^T u for every trajectory at the states y (holomorphic; host arrays)."""
        fa = (rtcc_field_t * self.ntraj)(*fields)
        tms = _as_c(times)
        y = np.ascontiguousarray(y, dtype=complex)
        u = np.ascontiguousarray(u, dtype=complex)
        assert y.shape == u.shape == (self.ntraj, self.ns)
        out = np.zeros_like(y)
        _check(_lib.rtcc_rhs_vjp(self.h, _ptr(y), fa, _ptr(tms), _ptr(u), _ptr(out)))
        return out

    def dipole(self):
        out = np.zeros((self.ntraj, 3), complex)
        _check(_lib.rtcc_dipole(self.h, _ptr(out)))
        return out

    def propagate(self, fields, integ, max_out, t_out=None, mu_out=None):
        fa = (rtcc_field_t * self.ntraj)(*fields)
        if t_out is None:
            t_out = np.zeros((self.ntraj, max_out))
            mu_out = np.zeros((self.ntraj, max_out, 3), complex)
        n_out = np.zeros(self.ntraj, np.int32)
        _check(_lib.rtcc_propagate(self.h, fa, C.byref(integ), max_out, _ptr(t_out), _ptr(mu_out),
                                   n_out.ctypes.data_as(_ip)))
        return t_out, mu_out, n_out

    def propagate_vjp(self, fields, hstep, nsteps, w, ckpt_every=25):
        """(J[z], dJ/d(E0, omega, sigma)[z]) by the checkpointed discrete adjoint of RK4."""
        fa = (rtcc_field_t * self.ntraj)(*fields)
        w = _as_c(w).reshape(nsteps + 1, 3)
        grad = np.zeros((self.ntraj, 3))
        J = np.zeros(self.ntraj)
        _check(_lib.rtcc_propagate_vjp(self.h, fa, hstep, nsteps, _ptr(w), ckpt_every, _ptr(grad), _ptr(J)))
        return J, grad

    def last_stats(self):
        """(accepted steps, rejected attempts, rhs evaluations, kernel launches) of the last propagate."""
        a, r, e, n = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_longlong()
        _check(_lib.rtcc_last_stats(self.h, C.byref(a), C.byref(r), C.byref(e), C.byref(n)))
        return a.value, r.value, e.value, n.value

    def profile_start(self):
        _check(_lib.rtcc_profile(self.h, 1, None))

    def profile_stop(self):
        p = rtcc_profile_t()
        _check(_lib.rtcc_profile(self.h, 0, C.byref(p)))
        return {KERNEL_CLASSES[k]: {"launches": p.launches[k], "ms": p.ms[k], "flops": p.flops[k],
                                    "bytes": p.bytes[k]} for k in range(8)}


def rtcc_spectrum(t, mu_re, field, omegas, kappa=0.0, gamma=0.01, dt=0.0):
    t, mu_re, omegas = _as_c(t), _as_c(mu_re), _as_c(omegas)
    I = np.zeros(len(omegas))
    _check(_lib.rtcc_spectrum(_ptr(t), _ptr(mu_re), len(t), C.byref(field), kappa, gamma, dt, _ptr(omegas),
                              len(omegas), _ptr(I)))
    return I


def rtcc_spectrum_pade(t, mu_re, field, omegas, kappa=0.0, gamma=0.01):
    """Pade-accelerated spectrum of uniformly spaced samples (at most 1025)."""
    t, mu_re, omegas = _as_c(t), _as_c(mu_re), _as_c(omegas)
    I = np.zeros(len(omegas))
    _check(_lib.rtcc_spectrum_pade(_ptr(t), _ptr(mu_re), len(t), C.byref(field), kappa, gamma, _ptr(omegas),
                                   len(omegas), _ptr(I)))
    return I


def rtcc_selftest_timeout(seconds):
    """Returns the status of a bounded device wait on a flag that nothing sets (expects TIMEOUT)."""
    code = _lib.rtcc_selftest_timeout(float(seconds))
    return STATUS.get(code, str(code))


def rtcc_selftest_gemm(prec, A, B):
    """C[b] = A[b] @ B[b]^T through the library's GEMM path (A: batch x M x K, B: batch x N x K,
    real or complex numpy arrays)."""
    ac, bc = np.iscomplexobj(A), np.iscomplexobj(B)
    A = np.ascontiguousarray(A, dtype=complex if ac else np.float64)
    B = np.ascontiguousarray(B, dtype=complex if bc else np.float64)
    nb, M, K = A.shape
    N = B.shape[1]
    Cm = np.zeros((nb, M, N), dtype=complex if (ac or bc) else np.float64)
    _check(_lib.rtcc_selftest_gemm(int(prec), int(ac) | (int(bc) << 1), nb, M, N, K, _ptr(A), _ptr(B), _ptr(Cm)))
    return Cm


def _check_noalloc_args(A, B, Cout):
    """The checks rtcc_gemm_noalloc needs before it hands raw device pointers to the library:
    dtypes, shapes, contiguity and one CUDA device for all three tensors (ValueError otherwise)."""
    import torch
    for name, t in (("A", A), ("B", B), ("Cout", Cout)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype not in (torch.float64, torch.complex128):
            raise ValueError(f"{name} must be float64 or complex128, not {t.dtype}")
        if t.dim() != 3:
            raise ValueError(f"{name} must have three dimensions (batch, rows, K or columns)")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    nb, M, K = A.shape
    N = B.shape[1]
    if tuple(B.shape) != (nb, N, K):
        raise ValueError(f"B has shape {tuple(B.shape)}, expected (batch, N, K) = ({nb}, N, {K})")
    if tuple(Cout.shape) != (nb, M, N):
        raise ValueError(f"Cout has shape {tuple(Cout.shape)}, expected ({nb}, {M}, {N})")
    want = torch.complex128 if (A.is_complex() or B.is_complex()) else torch.float64
    if Cout.dtype != want:
        raise ValueError(f"Cout must be {want} for these inputs, not {Cout.dtype}")
    if min(nb, M, N, K) < 1:
        raise ValueError("empty GEMM")
    devs = {t.device for t in (A, B, Cout)}
    if len(devs) != 1 or next(iter(devs)).type != "cuda":
        raise ValueError(f"A, B and Cout must be on one CUDA device, got {sorted(str(d) for d in devs)}")
    return nb, M, N, K


def rtcc_gemm_noalloc(prec, A, B, Cout, stream=None):
    """C[b] = A[b] @ B[b]^T on the GPU without any allocation by the library.

    A (batch x M x K), B (batch x N x K) and Cout (batch x M x N) are contiguous CUDA tensors on
    one device, of dtype float64 or complex128 (Cout complex128 when either input is complex);
    Cout is overwritten.  For callers that own all device memory themselves: the library's
    scratch is a fixed static device array.  Bad dtypes, shapes or devices raise ValueError
    before anything reaches the device.
    """
    nb, M, N, K = _check_noalloc_args(A, B, Cout)
    ac, bc = A.is_complex(), B.is_complex()
    st = stream.cuda_stream if stream is not None else 0
    _check(_lib.rtcc_gemm_noalloc(int(prec), int(ac) | (int(bc) << 1), nb, M, N, K, _ptr(A), _ptr(B), _ptr(Cout),
                                  C.c_void_p(st)))
    return Cout


def make_objective(handle, hstep, nsteps, w, ckpt_every=25, field_kw=None):
    """torch.autograd.Function: theta = (E0, omega, sigma) -> J = sum_n sum_x w[n][x] Re mu_x(t_n)
    for trajectory 0 of `handle`, differentiated by rtcc_propagate_vjp.  The state at the start
    (the handle's current state) is restored by the library after every call."""
    import torch
    kw = dict(field_kw or {})

    class _Objective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta):
            e0, om, sg = (float(x) for x in theta.detach().cpu())
            f = make_field(E0=e0, omega=om, sigma=sg, **kw)
            J, g = handle.propagate_vjp([f] * handle.ntraj, hstep, nsteps, w, ckpt_every)
            ctx.save_for_backward(torch.tensor(g[0], dtype=theta.dtype))
            return torch.tensor(J[0], dtype=theta.dtype)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout * g

    return _Objective.apply
