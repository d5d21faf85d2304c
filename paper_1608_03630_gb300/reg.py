"""Thin Python binding of libreg.so (the C-ABI in include/reg.h).

Argument marshalling only: every step of the registration path runs in the
library's CUDA kernels and cuFFT.  Fields are torch CUDA float32 tensors,
contiguous, scalar fields shaped (n1, n2, n3) and vector fields (3, n1, n2, n3);
the binding passes their device pointers and the current torch stream.  If
the library is not built, loading raises -- there is no other code path.
"""

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, 'libreg.so')

H1, H2, H1DIV = 1, 2, 3
KINDS = {'H1': H1, 'H2': H2, 'H1DIV': H1DIV}
FP32, MIXED_BF16 = 0, 1
PHASES = ('departure', 'state', 'adjoint', 'incstate', 'incadj', 'interp', 'fft',
          'spectral', 'blas', 'other', 'deriv')


class RegError(RuntimeError):
    def __init__(self, status, message):
        super().__init__('%s: %s' % (status_name(status), message))
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [('gtol', ctypes.c_double), ('max_gn', ctypes.c_int),
                ('max_pcg', ctypes.c_int), ('forcing', ctypes.c_int),
                ('armijo_c', ctypes.c_double), ('armijo_shrink', ctypes.c_double),
                ('armijo_max', ctypes.c_int), ('use_graph', ctypes.c_int),
                ('verbose', ctypes.c_int), ('gnorm_ref', ctypes.c_double),
                ('precond_shift', ctypes.c_double), ('beta_start', ctypes.c_double),
                ('beta_factor', ctypes.c_double), ('coarse_factor', ctypes.c_int),
                ('coarse_tol', ctypes.c_double), ('coarse_max', ctypes.c_int),
                ('coarse_nt', ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [('gn_iters', ctypes.c_int), ('pcg_iters', ctypes.c_int),
                ('matvecs', ctypes.c_int), ('objective_evals', ctypes.c_int),
                ('gradient_evals', ctypes.c_int), ('line_search_failed', ctypes.c_int),
                ('negative_curvature', ctypes.c_int),
                ('J0', ctypes.c_double), ('J', ctypes.c_double),
                ('gnorm0', ctypes.c_double), ('gnorm', ctypes.c_double),
                ('gnorm_rel', ctypes.c_double), ('mismatch_rel', ctypes.c_double),
                ('ms_total', ctypes.c_double), ('stages', ctypes.c_int),
                ('coarse_matvecs', ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


NPHASES = 11


class Timing(ctypes.Structure):
    _fields_ = [('ms', ctypes.c_double * NPHASES), ('launches', ctypes.c_longlong * NPHASES),
                ('bytes', ctypes.c_double * NPHASES)]

    def as_dict(self):
        return {p: dict(ms=self.ms[i], launches=self.launches[i], bytes=self.bytes[i])
                for i, p in enumerate(PHASES)}


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    'reg_create': [_I, _I, _I, _I, _D, _I, _I, ctypes.POINTER(_P)],
    'reg_destroy': [_P],
    'reg_set_stream': [_P, _P],
    'reg_set_precision': [_P, _I],
    'reg_set_hessian': [_P, _I],
    'reg_set_persistent': [_P, _I],
    'reg_set_images': [_P, _P, _P, _I],
    'reg_objective': [_P, _P, ctypes.POINTER(_D)],
    'reg_gradient': [_P, _P, _P, ctypes.POINTER(_D)],
    'reg_hessian_matvec': [_P, _P, _P],
    'reg_precond_apply': [_P, _P, _P],
    'reg_gradient_spectral': [_P, _P, _P, ctypes.POINTER(_D)],
    'reg_hessian_matvec_spectral': [_P, _P, _P],
    'reg_solve_opts_default': [ctypes.POINTER(SolveOpts)],
    'reg_set_beta': [_P, _D],
    'reg_twolevel_setup': [_P, _I, _P],
    'reg_twolevel_setup_nt': [_P, _I, _I, _P],
    'reg_twolevel_apply': [_P, _P, _P, _D, _I, ctypes.POINTER(_I)],
    'reg_solve': [_P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats)],
    'reg_solve_host': [_P, _P, _P, _I, _P, ctypes.POINTER(SolveOpts),
                       ctypes.POINTER(SolveStats)],
    'reg_departure': [_P, _P, _P, _P],
    'reg_interp': [_P, _P, _I, _P, _P],
    'reg_state_transport': [_P, _P, _P, _P],
    'reg_spectral_grad': [_P, _P, _P],
    'reg_spectral_div': [_P, _P, _P],
    'reg_leray': [_P, _P, _P],
    'reg_apply_regularisation': [_P, _P, _P],
    'reg_gaussian_smooth': [_P, _P, _P, _D, _D, _D],
    'reg_inner': [_P, _P, _P, ctypes.c_size_t, ctypes.POINTER(_D)],
    'reg_set_timing': [_P, _I],
    'reg_set_tile': [_P, _I, _I],
    'reg_get_tile': [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    'reg_set_staging': [_P, _I],
    'reg_debug_inject': [_I, _I],
    'reg_get_timing': [_P, ctypes.POINTER(Timing)],
    'reg_get_coarse_timing': [_P, ctypes.POINTER(Timing)],
    'reg_get_coarse_tile': [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    'reg_set_coarse_tile': [_P, _I, _I],
    'reg_set_dependent_launch': [_I],
    'reg_autotune': [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    'reg_batch_create': [_I, _P, _I, _D, _I, _I, _I, ctypes.POINTER(_P)],
    'reg_batch_destroy': [_P],
    'reg_batch_set_mode': [_P, _I],
    'reg_batch_graphs_launched': [_P, ctypes.POINTER(_I)],
    'reg_batch_solve': [_P, _P, _P, _P, _I, _I, ctypes.POINTER(SolveOpts), _P, _P, _P],
    'reg_spectral_resample': [_P, _P, _I, _P, _P, _P],
    'reg_deformation': [_P, _P, _P],
    'reg_jacobian_det': [_P, _P, _P],
    'reg_unet_create': [_I, _I, _P, _I, _I, ctypes.POINTER(_P)],
    'reg_unet_destroy': [_P],
    'reg_unet_set_stream': [_P, _P],
    'reg_unet_set_mma': [_P, _I],
    'reg_unet_param_count': [_P, ctypes.POINTER(ctypes.c_size_t)],
    'reg_unet_set_params': [_P, _P],
    'reg_unet_get_params': [_P, _P],
    'reg_unet_forward': [_P, _P, _P],
    'reg_unet_gradient': [_P, _P, _P, ctypes.POINTER(_D), _P],
    'reg_unet_train_step': [_P, _P, _P, ctypes.c_float, ctypes.POINTER(_D)],
}


def lib():
    """Load libreg.so once (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError('libreg.so is not built (%s); run '
                              '`python -c "import __graft_entry__ as g; g.build()"`' % LIB_PATH)
        l = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        l.reg_last_error.argtypes = [_P]
        l.reg_last_error.restype = ctypes.c_char_p
        l.reg_state_transport_noalloc.argtypes = [_I, _I, _I, _I, _P, _P, _P, _P]
        l.reg_state_transport_noalloc.restype = ctypes.c_int
        l.reg_unet_last_error.argtypes = [_P]
        l.reg_unet_last_error.restype = ctypes.c_char_p
        l.reg_status_string.argtypes = [_I]
        l.reg_status_string.restype = ctypes.c_char_p
        _lib = l
    return _lib


def status_name(s):
    try:
        return lib().reg_status_string(s).decode()
    except Exception:
        return 'status %d' % s


INJECT = {'none': 0, 'alloc': 1, 'cufft_plan': 2, 'nan_image': 3, 'stage_timeout': 4}


def debug_inject(what, after=0):
    """Arm one host-side fault injection (reg_debug_inject): 'alloc' or
    'cufft_plan' fails the (after + 1)-th device allocation or cuFFT plan of
    reg_create; 'nan_image' puts a NaN into the next reg_set_images;
    'stage_timeout' makes the next TMA-staged interpolation launch wait for a
    copy it never issued, so its bounded waits run out; 'none' disarms."""
    s = lib().reg_debug_inject(INJECT[what], int(after))
    if s != 0:
        raise RegError(s, 'reg_debug_inject(%r, %r)' % (what, after))


def _ptr(t, shape=None, what='tensor'):
    if not isinstance(t, torch.Tensor):
        raise TypeError('%s must be a torch tensor' % what)
    if t.device.type != 'cuda' or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError('%s must be a contiguous CUDA float32 tensor' % what)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError('%s has shape %s, expected %s' % (what, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


def set_dependent_launch(on):
    """Process-wide: programmatic dependent launches of the PCG-path kernels
    (True, the default) or ordinary launches (reg_set_dependent_launch)."""
    s = lib().reg_set_dependent_launch(1 if on else 0)
    if s != 0:
        raise RegError(s, 'reg_set_dependent_launch failed')


def state_transport_noalloc(rho0, d_fwd, rho1, nt, stream=None):
    """reg_state_transport_noalloc: rho1 = rho(t_nt) from rho0 with the
    points d_fwd, with no allocation and no context (see include/reg.h).
    The three tensors must be on one device; the call runs with that device
    current, on `stream` (default: that device's current stream)."""
    shape = tuple(rho0.shape)
    devs = {t.device for t in (rho0, d_fwd, rho1)}
    if len(devs) != 1:
        raise ValueError('rho0, d_fwd and rho1 must be on one device, got %s' % sorted(map(str, devs)))
    device = rho0.device
    with torch.cuda.device(device):
        if stream is None:
            stream = torch.cuda.current_stream(device)
        s = lib().reg_state_transport_noalloc(shape[0], shape[1], shape[2], int(nt),
                                              _ptr(rho0, shape, 'rho0'),
                                              _ptr(d_fwd, (3,) + shape, 'd_fwd'),
                                              _ptr(rho1, shape, 'rho1'),
                                              ctypes.c_void_p(stream.cuda_stream))
    if s != 0:
        raise RegError(s, 'reg_state_transport_noalloc failed')


class Registration:
    """One registration context (reg_create ... reg_destroy)."""

    def __init__(self, shape, nt, beta, kind='H2', incompressible=False, precision='fp32',
                 stream=None):
        self.shape = tuple(int(s) for s in shape)
        self.nt = int(nt)
        self.n = self.shape[0] * self.shape[1] * self.shape[2]
        self._ctx = ctypes.c_void_p()
        L = lib()
        s = L.reg_create(self.shape[0], self.shape[1], self.shape[2], self.nt, float(beta),
                         KINDS[kind] if isinstance(kind, str) else int(kind),
                         1 if incompressible else 0, ctypes.byref(self._ctx))
        if s != 0:
            raise RegError(s, L.reg_last_error(None).decode())
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._call('reg_set_stream', ctypes.c_void_p(stream.cuda_stream))
        if precision not in ('fp32', 'mixed_bf16'):
            raise ValueError(precision)
        if precision == 'mixed_bf16':
            self._call('reg_set_precision', MIXED_BF16)

    # -- plumbing ---------------------------------------------------------
    def _call(self, name, *args):
        s = getattr(lib(), name)(self._ctx, *args)
        if s != 0:
            raise RegError(s, lib().reg_last_error(self._ctx).decode())
        return s

    def close(self):
        if self._ctx and self._ctx.value:
            lib().reg_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def vshape(self):
        return (3,) + self.shape

    def _new(self, shape):
        return torch.empty(shape, device='cuda', dtype=torch.float32)

    # -- API --------------------------------------------------------------
    def set_beta(self, beta):
        """Regularisation weight beta > 0 (reg_set_beta)."""
        self._call('reg_set_beta', float(beta))

    def set_persistent(self, on):
        """Small grids: one persistent launch per PCG matvec transport (True)
        or the time steps one by one (False, the default)."""
        self._call('reg_set_persistent', 1 if on else 0)

    def set_hessian(self, full_newton):
        """True: full Newton Hessian (Eq. hessian with the lam terms);
        False: Gauss-Newton (the default)."""
        self._call('reg_set_hessian', 1 if full_newton else 0)

    def set_images(self, rho_T, rho_R, presmooth=False):
        self._call('reg_set_images', _ptr(rho_T, self.shape, 'rho_T'),
                   _ptr(rho_R, self.shape, 'rho_R'), 1 if presmooth else 0)

    def objective(self, v):
        J = ctypes.c_double()
        self._call('reg_objective', _ptr(v, self.vshape, 'v'), ctypes.byref(J))
        return J.value

    def gradient(self, v, out=None):
        g = self._new(self.vshape) if out is None else out
        J = ctypes.c_double()
        self._call('reg_gradient', _ptr(v, self.vshape, 'v'), _ptr(g, self.vshape, 'g'),
                   ctypes.byref(J))
        return g, J.value

    def hessian_matvec(self, vt, out=None):
        o = self._new(self.vshape) if out is None else out
        self._call('reg_hessian_matvec', _ptr(vt, self.vshape, 'vt'), _ptr(o, self.vshape, 'Hvt'))
        return o

    @property
    def sshape(self):
        """Shape of a vector field's normalised half spectrum as a complex64
        tensor: (3, n1, n2, n3 // 2 + 1)."""
        return (3, self.shape[0], self.shape[1], self.shape[2] // 2 + 1)

    def _cptr(self, t, what):
        if not isinstance(t, torch.Tensor) or t.device.type != 'cuda' or \
                t.dtype != torch.complex64 or not t.is_contiguous() or \
                tuple(t.shape) != self.sshape:
            raise ValueError('%s must be a contiguous CUDA complex64 tensor of shape %s'
                             % (what, self.sshape))
        return ctypes.c_void_p(t.data_ptr())

    def gradient_spectral(self, v_hat, out=None):
        """(g_hat, J) from normalised half-spectrum coefficients v_hat
        (complex64 (3, n1, n2, n3 // 2 + 1)); reg_gradient_spectral."""
        g = torch.empty(self.sshape, device='cuda', dtype=torch.complex64) if out is None else out
        J = ctypes.c_double()
        self._call('reg_gradient_spectral', self._cptr(v_hat, 'v_hat'), self._cptr(g, 'g_hat'),
                   ctypes.byref(J))
        return g, J.value

    def hessian_matvec_spectral(self, vt_hat, out=None):
        """Hvt_hat from the coefficients vt_hat; reg_hessian_matvec_spectral."""
        o = torch.empty(self.sshape, device='cuda', dtype=torch.complex64) if out is None else out
        self._call('reg_hessian_matvec_spectral', self._cptr(vt_hat, 'vt_hat'),
                   self._cptr(o, 'Hvt_hat'))
        return o

    def twolevel_setup(self, factor, v_hat, coarse_nt=0):
        """Coarse grid n / factor, restricted images, coarse Hessian (with
        coarse_nt time steps, 0: the context's) at the restriction of v_hat
        (reg_twolevel_setup_nt)."""
        self._call('reg_twolevel_setup_nt', int(factor), int(coarse_nt),
                   self._cptr(v_hat, 'v_hat'))

    def twolevel_apply(self, r_hat, inner_tol=0.1, inner_max=10, out=None):
        """(z_hat, inner iterations) = two-level M^-1 r_hat (reg_twolevel_apply)."""
        o = torch.empty(self.sshape, device='cuda', dtype=torch.complex64) if out is None else out
        it = ctypes.c_int()
        self._call('reg_twolevel_apply', self._cptr(r_hat, 'r_hat'), self._cptr(o, 'z_hat'),
                   float(inner_tol), int(inner_max), ctypes.byref(it))
        return o, it.value

    def precond(self, r, out=None):
        o = self._new(self.vshape) if out is None else out
        self._call('reg_precond_apply', _ptr(r, self.vshape, 'r'), _ptr(o, self.vshape, 'z'))
        return o

    @staticmethod
    def default_opts():
        o = SolveOpts()
        lib().reg_solve_opts_default(ctypes.byref(o))
        return o

    def _opts(self, kw):
        o = self.default_opts()
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def solve(self, v, **opts):
        """Solve in place from the initial guess v; returns (status, stats)."""
        st = SolveStats()
        s = lib().reg_solve(self._ctx, _ptr(v, self.vshape, 'v'), ctypes.byref(self._opts(opts)),
                            ctypes.byref(st))
        if s not in (0, 7):
            raise RegError(s, lib().reg_last_error(self._ctx).decode())
        return s, st.as_dict()

    def solve_host(self, rho_T_host, rho_R_host, v_host, presmooth=False, **opts):
        """Same solve through host (CPU) float32 tensors; v_host is updated."""
        for t, nm in ((rho_T_host, 'rho_T'), (rho_R_host, 'rho_R'), (v_host, 'v')):
            if t.device.type != 'cpu' or t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError('%s must be a contiguous CPU float32 tensor' % nm)
        st = SolveStats()
        s = lib().reg_solve_host(self._ctx, ctypes.c_void_p(rho_T_host.data_ptr()),
                                 ctypes.c_void_p(rho_R_host.data_ptr()), 1 if presmooth else 0,
                                 ctypes.c_void_p(v_host.data_ptr()),
                                 ctypes.byref(self._opts(opts)), ctypes.byref(st))
        if s not in (0, 7):
            raise RegError(s, lib().reg_last_error(self._ctx).decode())
        return s, st.as_dict()

    def departure(self, v):
        df, da = self._new(self.vshape), self._new(self.vshape)
        self._call('reg_departure', _ptr(v, self.vshape, 'v'), _ptr(df), _ptr(da))
        return df, da

    def interp(self, field, disp, out=None):
        nf = 1 if field.dim() == 3 else field.shape[0]
        o = torch.empty_like(field) if out is None else out
        self._call('reg_interp', _ptr(field, None, 'field'), nf, _ptr(disp, self.vshape, 'disp'),
                   _ptr(o, tuple(field.shape), 'out'))
        return o

    def state_transport(self, rho0, d_fwd):
        hist = self._new((self.nt + 1,) + self.shape)
        self._call('reg_state_transport', _ptr(rho0, self.shape, 'rho0'),
                   _ptr(d_fwd, self.vshape, 'd_fwd'), _ptr(hist))
        return hist

    def deformation(self, v, out=None):
        """u = y(x, 1) - x of the deformation map of v (reg_deformation)."""
        u = self._new(self.vshape) if out is None else out
        self._call('reg_deformation', _ptr(v, self.vshape, 'v'), _ptr(u, self.vshape, 'u'))
        return u

    def jacobian_det(self, u, out=None):
        """det(I + grad u) (reg_jacobian_det)."""
        d = self._new(self.shape) if out is None else out
        self._call('reg_jacobian_det', _ptr(u, self.vshape, 'u'), _ptr(d, self.shape, 'det'))
        return d

    def spectral_grad(self, f):
        o = self._new(self.vshape)
        self._call('reg_spectral_grad', _ptr(f, self.shape, 'f'), _ptr(o))
        return o

    def spectral_div(self, v):
        o = self._new(self.shape)
        self._call('reg_spectral_div', _ptr(v, self.vshape, 'v'), _ptr(o))
        return o

    def leray(self, v, out=None):
        o = self._new(self.vshape) if out is None else out
        self._call('reg_leray', _ptr(v, self.vshape, 'v'), _ptr(o, self.vshape, 'out'))
        return o

    def apply_regularisation(self, v):
        o = self._new(self.vshape)
        self._call('reg_apply_regularisation', _ptr(v, self.vshape, 'v'), _ptr(o))
        return o

    def gaussian_smooth(self, f, sigma):
        o = self._new(self.shape)
        self._call('reg_gaussian_smooth', _ptr(f, self.shape, 'f'), _ptr(o), float(sigma[0]),
                   float(sigma[1]), float(sigma[2]))
        return o

    def inner(self, a, b):
        out = ctypes.c_double()
        self._call('reg_inner', _ptr(a), _ptr(b), ctypes.c_size_t(a.numel()), ctypes.byref(out))
        return out.value

    def set_tile(self, k, wy):
        self._call('reg_set_tile', int(k), int(wy))

    def set_staging(self, tma):
        """True: stage interpolation boxes with one TMA copy per block where
        the grid allows; False: per-thread cp.async copies (same results)."""
        self._call('reg_set_staging', 1 if tma else 0)

    def get_tile(self):
        k, wy = ctypes.c_int(), ctypes.c_int()
        self._call('reg_get_tile', ctypes.byref(k), ctypes.byref(wy))
        return k.value, wy.value

    def autotune(self):
        k, wy = ctypes.c_int(), ctypes.c_int()
        self._call('reg_autotune', ctypes.byref(k), ctypes.byref(wy))
        return k.value, wy.value

    def set_timing(self, on):
        self._call('reg_set_timing', 1 if on else 0)

    def get_timing(self):
        t = Timing()
        self._call('reg_get_timing', ctypes.byref(t))
        return t.as_dict()

    def get_coarse_timing(self):
        """Per-phase figures of the two-level preconditioner's coarse grid."""
        t = Timing()
        self._call('reg_get_coarse_timing', ctypes.byref(t))
        return t.as_dict()

    def set_coarse_tile(self, k, wy):
        """The coarse grid's tile: (0, 0) autotuned (default), else as given
        (reg_set_coarse_tile)."""
        self._call('reg_set_coarse_tile', int(k), int(wy))

    def get_coarse_tile(self):
        """(k, wy) of the two-level preconditioner's coarse grid ((0, 0)
        without one)."""
        k, wy = ctypes.c_int(), ctypes.c_int()
        self._call('reg_get_coarse_tile', ctypes.byref(k), ctypes.byref(wy))
        return k.value, wy.value


class Batch:
    """reg_batch_*: independent pairs of uneven sizes solved concurrently."""

    def __init__(self, shapes, nt, beta, kind='H2', incompressible=False, precision='fp32'):
        self.shapes = [tuple(int(x) for x in s) for s in shapes]
        dims = (ctypes.c_int * (3 * len(shapes)))(*[x for s in self.shapes for x in s])
        self._b = ctypes.c_void_p()
        s = lib().reg_batch_create(len(shapes), ctypes.cast(dims, ctypes.c_void_p), int(nt),
                                   float(beta), KINDS[kind], 1 if incompressible else 0,
                                   MIXED_BF16 if precision == 'mixed_bf16' else FP32,
                                   ctypes.byref(self._b))
        if s != 0:
            raise RegError(s, lib().reg_last_error(None).decode())

    def set_mode(self, one_graph):
        """True: lockstep Newton steps, one PCG graph per step for all pairs
        (default); False: whole solves on worker threads."""
        s = lib().reg_batch_set_mode(self._b, 0 if one_graph else 1)
        if s != 0:
            raise RegError(s, 'reg_batch_set_mode')

    def graphs_launched(self):
        n = ctypes.c_int()
        lib().reg_batch_graphs_launched(self._b, ctypes.byref(n))
        return n.value

    def solve(self, vs, rho_Ts, rho_Rs, presmooth=True, autotune=True, **opts):
        """Solve all pairs in place; returns (statuses, stats dicts, latencies ms)."""
        n = len(self.shapes)
        ptrs = lambda ts, nm: (ctypes.c_void_p * n)(*[_ptr(t, None, nm).value for t in ts])
        o = Registration.default_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        stats = (SolveStats * n)()
        lat = (ctypes.c_double * n)()
        st = (ctypes.c_int * n)()
        torch.cuda.synchronize()
        s = lib().reg_batch_solve(self._b, ptrs(vs, 'v'), ptrs(rho_Ts, 'rho_T'),
                                  ptrs(rho_Rs, 'rho_R'), 1 if presmooth else 0,
                                  1 if autotune else 0, ctypes.byref(o),
                                  ctypes.cast(stats, ctypes.c_void_p),
                                  ctypes.cast(lat, ctypes.c_void_p),
                                  ctypes.cast(st, ctypes.c_void_p))
        if s != 0:
            raise RegError(s, 'reg_batch_solve failed')
        return list(st), [x.as_dict() for x in stats], list(lat)

    def close(self):
        if self._b and self._b.value:
            lib().reg_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spectral_resample(x, shape_out, stream=None):
    """reg_spectral_resample: Fourier resampling of x (c, n1, n2, n3) or
    (n1, n2, n3) to the grid shape_out; returns a new CUDA tensor."""
    scalar = x.dim() == 3
    xs = x.unsqueeze(0) if scalar else x
    c = xs.shape[0]
    nin = (ctypes.c_int * 3)(*xs.shape[1:])
    nout = (ctypes.c_int * 3)(*[int(v) for v in shape_out])
    out = torch.empty((c,) + tuple(int(v) for v in shape_out), device=x.device,
                      dtype=torch.float32)
    if stream is None:
        stream = torch.cuda.current_stream()
    s = lib().reg_spectral_resample(ctypes.cast(nin, _P), ctypes.cast(nout, _P), int(c),
                                    _ptr(xs, None, 'x'), _ptr(out, None, 'out'),
                                    ctypes.c_void_p(stream.cuda_stream))
    if s != 0:
        raise RegError(s, 'reg_spectral_resample failed')
    return out[0] if scalar else out


class UNet:
    """reg_unet_*: the 3-D U-Net of the learned initial velocity.

    x is a CUDA float32 tensor (cin, R, R, R); predictions and targets are
    (cout, R, R, R).  Parameters are a flat float32 numpy array in the order
    of include/reg.h (per layer: weights [kz][ky][kx][cin][cout], bias)."""

    def __init__(self, R, channels=(16, 32, 64, 128), cin=2, cout=3):
        self.R, self.channels, self.cin, self.cout = int(R), tuple(channels), cin, cout
        ch = (ctypes.c_int * len(self.channels))(*self.channels)
        self._u = ctypes.c_void_p()
        s = lib().reg_unet_create(self.R, len(self.channels), ctypes.cast(ch, _P), cin, cout,
                                  ctypes.byref(self._u))
        if s != 0:
            raise RegError(s, 'reg_unet_create failed')
        n = ctypes.c_size_t()
        self._call('reg_unet_param_count', ctypes.byref(n))
        self.nparams = n.value

    def _call(self, name, *args):
        lib().reg_unet_set_stream(self._u, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        s = getattr(lib(), name)(self._u, *args)
        if s != 0:
            raise RegError(s, lib().reg_unet_last_error(self._u).decode())

    def set_mma(self, tcgen05):
        """True: forward 3x3x3 convolutions on tcgen05 where they fit; False:
        the wmma path for every layer."""
        self._call('reg_unet_set_mma', 1 if tcgen05 else 0)

    def layer_shapes(self):
        """(name, weight shape, bias shape) per layer, in parameter order."""
        ch, L = self.channels, len(self.channels)
        out, prev = [], self.cin
        for l in range(L):
            out.append(('enc%d.0' % l, (3, 3, 3, prev, ch[l]), (ch[l],)))
            out.append(('enc%d.1' % l, (3, 3, 3, ch[l], ch[l]), (ch[l],)))
            prev = ch[l]
        for l in range(L - 2, -1, -1):
            out.append(('dec%d.0' % l, (3, 3, 3, ch[l + 1] + ch[l], ch[l]), (ch[l],)))
            out.append(('dec%d.1' % l, (3, 3, 3, ch[l], ch[l]), (ch[l],)))
        out.append(('head', (1, 1, 1, ch[0], self.cout), (self.cout,)))
        return out

    def pack(self, params):
        """Flat float32 array from a dict {'name.w': ..., 'name.b': ...}."""
        import numpy as np
        parts = []
        for name, ws, bs in self.layer_shapes():
            parts.append(np.asarray(params[name + '.w'], dtype=np.float32).reshape(-1))
            parts.append(np.asarray(params[name + '.b'], dtype=np.float32).reshape(-1))
        flat = np.concatenate(parts)
        assert flat.size == self.nparams
        return flat

    def unpack(self, flat):
        import numpy as np
        out, o = {}, 0
        for name, ws, bs in self.layer_shapes():
            nw, nb = int(np.prod(ws)), int(np.prod(bs))
            out[name + '.w'] = flat[o:o + nw].reshape(ws)
            o += nw
            out[name + '.b'] = flat[o:o + nb].reshape(bs)
            o += nb
        return out

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparams
        self._call('reg_unet_set_params', a.ctypes.data_as(_P))

    def get_params(self):
        import numpy as np
        a = np.empty(self.nparams, dtype=np.float32)
        self._call('reg_unet_get_params', a.ctypes.data_as(_P))
        return a

    def _x(self, x):
        return _ptr(x, (self.cin, self.R, self.R, self.R), 'x')

    def forward(self, x, out=None):
        if out is None:
            out = torch.empty((self.cout, self.R, self.R, self.R), device=x.device)
        self._call('reg_unet_forward', self._x(x), _ptr(out, (self.cout,) + (self.R,) * 3, 'y'))
        return out

    def gradient(self, x, target):
        """(loss, flat FP32 gradient) of the mean squared error."""
        import numpy as np
        g = np.empty(self.nparams, dtype=np.float32)
        loss = ctypes.c_double()
        self._call('reg_unet_gradient', self._x(x),
                   _ptr(target, (self.cout,) + (self.R,) * 3, 'target'), ctypes.byref(loss),
                   g.ctypes.data_as(_P))
        return loss.value, g

    def train_step(self, x, target, lr, want_loss=True):
        loss = ctypes.c_double()
        self._call('reg_unet_train_step', self._x(x),
                   _ptr(target, (self.cout,) + (self.R,) * 3, 'target'), ctypes.c_float(lr),
                   ctypes.byref(loss) if want_loss else None)
        return loss.value if want_loss else None

    def close(self):
        if self._u and self._u.value:
            lib().reg_unet_destroy(self._u)
            self._u = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
