"""FP64 CPU oracle for the Gauss-Newton-Krylov registration hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
NumPy restatement of what the method computes (Mang, Gholami, Biros,
"Distributed-memory large deformation diffeomorphic 3D image registration",
SC16).  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The GPU library never imports it, and it
never imports the GPU library: the two share no code.

Every function follows a passage of the paper, cited in its docstring by
section and equation:

* ``spectral``  -- Fourier differentiation, Leray projection, regularisation
                   operators and the spectral preconditioner (Sec. III-B1,
                   Eq. (gradient), Sec. III-A).
* ``interp``    -- tricubic Lagrange interpolation (Sec. III-C2).
* ``transport`` -- RK2 semi-Lagrangian points and the four transport solves
                   (Eq. (sml-trajectory), Eq. (sml-advection), Algorithm 2).
* ``problem``   -- objective, gradient and Gauss-Newton Hessian matvec
                   (Eq. (varopt), Eq. (gradient), Eq. (hessian)).
* ``solver``    -- PCG (and flexible PCG), the inexact Gauss-Newton method
                   with Armijo line search, parameter continuation on beta
                   (Sec. III-A, Sec. IV-A3).
* ``precond``   -- the two-level (coarse-grid Hessian plus inverse
                   regularisation) preconditioner (Sec. I limitations,
                   Sec. III-A, Table 5).

Readings of places where the paper is silent or garbled are listed in each
function's docstring.  Floating point throughout is float64; FFTs are
``numpy.fft`` (a library primitive used as one step).
"""

from . import spectral, interp, transport, problem, solver, precond  # noqa: F401
