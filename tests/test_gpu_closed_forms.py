"""Closed forms of the discrete operators, checked on the GPU directly (no
oracle involved): a single Fourier mode put into one field makes the
right-hand side of Eqs. 1-3 pick out one stencil, whose response on the
periodic grid is known exactly -- the modified wavenumbers of the
sixth-order first and second derivatives and the factor of the diagonal
mixed derivative (Sec. 2, Sec. 3.1).  Each case runs on the isotropic path
(cubic grid, equal spacings) and on the anisotropic one (three different
spacings), for the TMA kernel, the plane-ring kernel and the packed-FP32
tile."""
import math

import numpy as np
import pytest

from tests.gpu_util import gpu_params
from tests.states import coords, k1_mod, k2sq_mod, kmix_mod

pytestmark = pytest.mark.gpu

AXES = "xyz"
SHAPES = [(32, 32, 32), (40, 24, 16)]  # (nx, ny, nz); box 2 pi on every axis
KERNELS = [("f64", 2, 0), ("f64", 1, 0), ("f32", 2, 0), ("f32", 1, 0), ("f32", 2, 7), ("f32", 2, 17), ("f32", 2, 25), ("f32", 2, 26)]
TOL = {"f64": 1e-12, "f32": 2e-5}
NU, EPS, U = 0.05, 0.1, 0.1


def rhs_of(shape, dtype, kernel, tile, q):
    from paper_2012_08758_b300.run import Run
    nx, ny, nz = shape
    run = Run(**gpu_params(nx=nx, ny=ny, nz=nz, cs=1.0, nu=NU, eta=NU, f0=0.0, dtype=dtype, kernel=kernel,
                           tile=tile))
    run.set_state(q)
    r = run.eval_rhs()
    run.close()
    return r


def grid(shape):
    nx, ny, nz = shape
    X, Y, Z = coords(nx, ny, nz)
    return (X, Y, Z), [2 * math.pi / n for n in shape]


@pytest.mark.parametrize("dtype,kernel,tile", KERNELS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_first_derivative_through_pressure_gradient(axis, shape, dtype, kernel, tile):
    """ln rho = eps sin(k x_a), u = A = 0: d u_a/dt = -cs^2 eps k1 cos(k x_a)
    exactly; every other component of the right-hand side vanishes."""
    C, h = grid(shape)
    k = 3
    q = np.zeros((7,) + C[0].shape)
    q[0] = EPS * np.sin(k * C[axis])
    got = rhs_of(shape, dtype, kernel, tile, q)
    want = np.zeros_like(got)
    want[1 + axis] = -EPS * k1_mod(k, h[axis]) * np.cos(k * C[axis])
    amp = EPS * k1_mod(k, h[axis])
    assert np.abs(got - want).max() <= TOL[dtype] * amp


@pytest.mark.parametrize("dtype,kernel,tile", KERNELS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("a,b", [(0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)])
def test_second_derivative_through_viscous_shear(a, b, shape, dtype, kernel, tile):
    """u_b = U sin(k x_a) (a shear wave, a != b): the advection and div u
    vanish exactly, so d u_b/dt = -nu k2^2 U sin(k x_a); the mixed terms of
    grad div u are zero up to rounding, the rest exactly."""
    C, h = grid(shape)
    k = 2
    q = np.zeros((7,) + C[0].shape)
    q[1 + b] = U * np.sin(k * C[a])
    got = rhs_of(shape, dtype, kernel, tile, q)
    want = np.zeros_like(got)
    want[1 + b] = -NU * k2sq_mod(k, h[a]) * U * np.sin(k * C[a])
    amp = NU * k2sq_mod(k, h[a]) * U
    assert np.abs(got - want).max() <= TOL[dtype] * amp


@pytest.mark.parametrize("dtype,kernel,tile", KERNELS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("a,b", [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)])
def test_mixed_derivative_through_grad_div(a, b, shape, dtype, kernel, tile):
    """u_b = U sin(k x_a) sin(l x_b), the other components zero: the only
    term of d u_a/dt is nu/3 (grad div u)_a = nu/3 D_ab u_b, which the
    diagonal stencil gives as nu/3 U cos(k x_a) cos(l x_b) kmix(k, l) exactly.
    Each pair exercises its own path: the x-y pair from the output plane,
    the x-z and y-z pairs from the accumulators filled plane by plane."""
    C, h = grid(shape)
    k, l = 2, 3
    q = np.zeros((7,) + C[0].shape)
    q[1 + b] = U * np.sin(k * C[a]) * np.sin(l * C[b])
    got = rhs_of(shape, dtype, kernel, tile, q)
    m = kmix_mod(k, l, h[a], h[b])
    want = NU / 3 * U * m * np.cos(k * C[a]) * np.cos(l * C[b])
    amp = NU / 3 * U * abs(m)
    assert np.abs(got[1 + a] - want).max() <= TOL[dtype] * amp
