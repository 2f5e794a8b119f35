"""ORACLE -- test infrastructure, not part of the product.

A plain, slow, FP64 CPU implementation of what arXiv 2401.02896 ("Particle-Wise
Higher-Order SPH Field Approximation for DVR") computes on the per-ray path:

* the SPH kernels (Sec. 1, eq. cubic-kernel, plus Wendland C2/C4 and a poly6 test
  kernel under the compact-support assumption of Sec. 1);
* the optimal even piecewise-polynomial approximation of the unit-particle ray
  restriction B_L(t) = w(sqrt(L^2+t^2)) for given knots (Sec. 3.3: basis A~_kd,
  Gram-Schmidt in lexicographic order, sum of projections) and for optimal knots
  (Sec. 3.4), tabulated over equidistant L (the look-up table of Sec. 3.1);
* the per-ray field as the sum of the particles' approximations, with each
  piece's localized coefficients obtained by direct summation of the
  overlapping contributions (Sec. 2 localized coefficients; Sec. 4.1 direct
  alternative) -- no recurrence, so no drift;
* classification and emission-absorption compositing (Sec. 1), evaluated
  exactly per piece;
* gradients (Conclusion: the scheme carries over to additive features): the
  perpendicular gradient as approximations of G_L = w'(rho)/rho on each table
  entry's knots, the along-ray gradient as the derivative of the field's pieces,
  and emission shaded by ka + kd |n . v|.
* the quantised fixed-point path (Sec. 4.2-4.4, module ``oracle.quant``): the
  quantisation error estimate and optimal quanta, quantised knots in exact
  integers, and the per-ray field of exact integer coefficients.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with ``paper_2401_02896_b300``.
Functions whose correctness has no independent pin say "parity unpinned" in
their docstring; at present every function here has at least one pin in
``tests/test_oracle_*.py``.
"""
from .core import (  # noqa: F401
    KERNELS,
    kernel_support,
    kernel_w,
    lut_build,
    lut_build_grad,
    kernel_dw_r,
    composite_piece_shaded,
    fixed_knots,
    ray_norm2,
    ray_integral,
    render,
    particle_amplitude,
    composite_piece,
    camera_ray,
    Camera,
    num_threads,
    set_threads,
    entry_knots,
    field_eval,
)
