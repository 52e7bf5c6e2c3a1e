"""Pins of the FP64 oracle against what the paper's discretisation fixes
(closed forms, exact discrete invariants, polynomial brute force), so the
oracle is trusted on evidence other than itself.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests.states import coords, k1_mod, k2sq_mod, kmix_mod, rk3_gain, zero_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Stencils: exactness on polynomials (Sec. 2, 6th-order finite differences)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p", range(0, 9))
def test_d1_polynomial_exactness(p):
    h, x0 = 0.1, 0.37
    line = [(x0 + s * h) ** p for s in range(-3, 4)]
    exact = p * x0 ** (p - 1) if p > 0 else 0.0
    got = O.stencil_d1(line, h)
    if p <= 6:
        assert got == pytest.approx(exact, rel=1e-10, abs=1e-10)
    else:  # order exactly 6: degree 7 is no longer exact
        assert abs(got - exact) > 1e-9


@pytest.mark.parametrize("p", range(0, 10))
def test_d2_polynomial_exactness(p):
    h, x0 = 0.1, -0.23
    line = [(x0 + s * h) ** p for s in range(-3, 4)]
    exact = p * (p - 1) * x0 ** (p - 2) if p > 1 else 0.0
    got = O.stencil_d2(line, h)
    if p <= 7:
        assert got == pytest.approx(exact, rel=1e-9, abs=1e-9)
    else:
        assert abs(got - exact) > 1e-8


@pytest.mark.parametrize("a,b", [(a, b) for a in range(0, 8) for b in range(0, 8) if a + b <= 9])
def test_dmix_polynomial_exactness(a, b):
    ha, hb, x0, y0 = 0.1, 0.07, 0.31, -0.44
    patch = np.array([[(x0 + sa * ha) ** a * (y0 + sb * hb) ** b for sa in range(-3, 4)]
                      for sb in range(-3, 4)])
    exact = a * b * x0 ** max(a - 1, 0) * y0 ** max(b - 1, 0) if a > 0 and b > 0 else 0.0
    got = O.stencil_dmix(patch, ha, hb)
    if a + b <= 7:
        assert got == pytest.approx(exact, rel=1e-9, abs=1e-9)
    elif a % 2 == 1 and b % 2 == 1:  # odd-odd degree 8 term is not exact
        assert abs(got - exact) > 1e-9


def test_dmix_uses_only_diagonals():
    """Perturbing an off-diagonal point of the patch changes nothing."""
    rng = np.random.default_rng(3)
    patch = rng.standard_normal((7, 7))
    base = O.stencil_dmix(patch, 0.1, 0.1)
    p2 = patch.copy()
    p2[3 + 1, 3 + 2] += 5.0  # (sa=2, sb=1): off the diagonals
    p2[3, 3 + 1] += 5.0      # (sa=1, sb=0): on an axis
    assert O.stencil_dmix(p2, 0.1, 0.1) == base


# --------------------------------------------------------------------------
# Periodic stencils: single Fourier modes at the modified wavenumbers
# --------------------------------------------------------------------------
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_periodic_d1_d2_modified_wavenumber(axis):
    n = (12, 10, 14)
    p = O.Params(nx=n[0], ny=n[1], nz=n[2])
    X, Y, Z = coords(*n)
    C = (X, Y, Z)[axis]
    h = 2 * math.pi / n[axis]
    k = 2
    f = np.sin(k * C + 0.3)
    d1 = O.d1(p, f, axis)
    d2 = O.d2(p, f, axis)
    np.testing.assert_allclose(d1, k1_mod(k, h) * np.cos(k * C + 0.3), atol=1e-12)
    np.testing.assert_allclose(d2, -k2sq_mod(k, h) * np.sin(k * C + 0.3), atol=1e-12)
    # derivatives across the other axes vanish identically
    for other in {0, 1, 2} - {axis}:
        assert np.abs(O.d1(p, f, other)).max() < 1e-13


@pytest.mark.parametrize("a,b", [(0, 1), (0, 2), (1, 2), (1, 0)])
def test_periodic_dmix_closed_form(a, b):
    n = (10, 12, 8)
    p = O.Params(nx=n[0], ny=n[1], nz=n[2])
    XYZ = coords(*n)
    ha, hb = 2 * math.pi / n[a], 2 * math.pi / n[b]
    k, l = 2, 1
    f = np.sin(k * XYZ[a]) * np.sin(l * XYZ[b])
    got = O.dmix(p, f, a, b)
    want = np.cos(k * XYZ[a]) * np.cos(l * XYZ[b]) * kmix_mod(k, l, ha, hb)
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_sixth_order_convergence():
    errs1, errs2 = [], []
    for n in (16, 32):
        p = O.Params(nx=n, ny=4, nz=4)
        X, _, _ = coords(n, 4, 4)
        f = np.sin(X)
        errs1.append(np.abs(O.d1(p, f, 0) - np.cos(X)).max())
        errs2.append(np.abs(O.d2(p, f, 0) + np.sin(X)).max())
    for e in (errs1, errs2):
        order = math.log2(e[0] / e[1])
        assert 5.9 < order < 6.1, order


# --------------------------------------------------------------------------
# Right-hand side: one probe per term of Eqs. 1-3
# --------------------------------------------------------------------------
N3 = (12, 10, 8)


def _p(**kw):
    base = dict(nx=N3[0], ny=N3[1], nz=N3[2], nu=0.0, eta=0.0, cs=1.3)
    base.update(kw)
    return O.Params(**base)


def _grid():
    return coords(*N3), [2 * math.pi / n for n in N3]


def test_rhs_pressure_term():
    """ln rho = eps sin(kx), u = A = 0: du_x/dt = -cs^2 eps k1 cos(kx)."""
    p = _p()
    (X, Y, Z), h = _grid()
    q = zero_state(*N3)
    eps, k = 0.2, 2
    q[0] = eps * np.sin(k * X)
    r = O.rhs(p, q)
    np.testing.assert_allclose(r[1], -p.cs ** 2 * eps * k1_mod(k, h[0]) * np.cos(k * X), atol=1e-12)
    assert np.abs(r[[0, 2, 3, 4, 5, 6]]).max() < 1e-13


def test_rhs_density_advection_and_divergence():
    """Uniform u advects ln rho; a compressive u_z gives -div u."""
    p = _p()
    (X, Y, Z), h = _grid()
    q = zero_state(*N3)
    eps = 0.1
    q[0] = eps * np.sin(X) + eps * np.cos(2 * Y)
    q[1], q[2] = 0.3, -0.2
    q[3] = 0.05 * np.sin(Z)
    r = O.rhs(p, q)
    want = (-(0.3 * eps * k1_mod(1, h[0]) * np.cos(X) - 0.2 * (-eps * k1_mod(2, h[1]) * np.sin(2 * Y)))
            - 0.05 * k1_mod(1, h[2]) * np.cos(Z))
    np.testing.assert_allclose(r[0], want, atol=1e-12)


def test_rhs_self_advection():
    """u = (a sin kz, 0, c): du_x/dt = -c a k1 cos kz (nu = 0)."""
    p = _p()
    (X, Y, Z), h = _grid()
    q = zero_state(*N3)
    a, c = 0.4, 0.7
    q[1] = a * np.sin(2 * Z)
    q[3] = c
    r = O.rhs(p, q)
    np.testing.assert_allclose(r[1], -c * a * k1_mod(2, h[2]) * np.cos(2 * Z), atol=1e-12)
    assert np.abs(r[2]).max() < 1e-13 and np.abs(r[3]).max() < 1e-13


def test_rhs_viscous_compressive_mode():
    """u_x = a sin(kx): nu (lap u + grad div u / 3) = -(4/3) nu a k2^2 sin(kx),
    plus the advection -u_x d_x u_x."""
    nu = 0.3
    p = _p(nu=nu)
    (X, Y, Z), h = _grid()
    q = zero_state(*N3)
    a, k = 0.2, 2
    q[1] = a * np.sin(k * X)
    r = O.rhs(p, q)
    want = (-(4.0 / 3.0) * nu * a * k2sq_mod(k, h[0]) * np.sin(k * X)
            - a * np.sin(k * X) * a * k1_mod(k, h[0]) * np.cos(k * X))
    np.testing.assert_allclose(r[1], want, atol=1e-12)


@pytest.mark.parametrize("i,j", [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)])
def test_rhs_grad_div_cross_terms(i, j):
    """u_j = a sin(k x_i) sin(l x_j): the only force on u_i is
    nu/3 d_i d_j u_j, through the mixed stencil."""
    nu = 0.6
    p = _p(nu=nu)
    XYZ, h = _grid()
    q = zero_state(*N3)
    a, k, l = 0.1, 1, 2
    q[1 + j] = a * np.sin(k * XYZ[i]) * np.sin(l * XYZ[j])
    r = O.rhs(p, q)
    want = nu / 3.0 * a * np.cos(k * XYZ[i]) * np.cos(l * XYZ[j]) * kmix_mod(k, l, h[i], h[j])
    np.testing.assert_allclose(r[1 + i], want, atol=1e-12)


def test_rhs_strain_times_density_gradient():
    """ln rho = eps sin(kx), shear u_y = a sin(kx): the 2 S.grad ln rho term
    adds nu a eps k1^2 cos^2(kx) to du_y/dt; S is traceless, so a
    compressive u_x gives S_xx = (2/3) d_x u_x."""
    nu = 0.5
    p = _p(nu=nu, cs=1.0)
    (X, Y, Z), h = _grid()
    k, eps, a = 1, 0.1, 0.3
    k1 = k1_mod(k, h[0])
    q = zero_state(*N3)
    q[0] = eps * np.sin(k * X)
    q[2] = a * np.sin(k * X)
    r = O.rhs(p, q)
    want_y = nu * (-a * k2sq_mod(k, h[0]) * np.sin(k * X) + a * eps * k1 ** 2 * np.cos(k * X) ** 2)
    np.testing.assert_allclose(r[2], want_y, atol=1e-12)
    # compressive: u_x = a sin(kx)
    q = zero_state(*N3)
    q[0] = eps * np.sin(k * X)
    q[1] = a * np.sin(k * X)
    r = O.rhs(p, q)
    ux, dux = a * np.sin(k * X), a * k1 * np.cos(k * X)
    g = eps * k1 * np.cos(k * X)
    want_x = (-ux * dux - g + nu * (-(4.0 / 3.0) * a * k2sq_mod(k, h[0]) * np.sin(k * X)
                                     + 2 * (2.0 / 3.0) * dux * g))
    np.testing.assert_allclose(r[1], want_x, atol=1e-12)


def test_rhs_lorentz_force_and_density_factor():
    """A = (0, 0, a sin kx): B = (0, -a k1 cos kx, 0), j = (0, 0, a k2^2 sin kx),
    j x B / rho = (a^2 k1 k2^2 sin cos / rho, 0, 0)."""
    p = _p()
    (X, Y, Z), h = _grid()
    q = zero_state(*N3)
    a, k, c = 0.3, 2, 0.4
    q[0] = c
    q[6] = a * np.sin(k * X)
    r = O.rhs(p, q)
    want = a * a * k1_mod(k, h[0]) * k2sq_mod(k, h[0]) * np.sin(k * X) * np.cos(k * X) / math.exp(c)
    np.testing.assert_allclose(r[1], want, atol=1e-12)
    assert np.abs(r[2]).max() < 1e-13 and np.abs(r[3]).max() < 1e-13


def test_rhs_induction_u_cross_b_and_resistivity():
    """u = (0, 0, U), A = (0, 0, a sin kx): dA_x/dt = U a k1 cos kx;
    dA_z/dt = -eta a k2^2 sin kx."""
    eta = 0.2
    p = _p(eta=eta)
    (X, Y, Z), h = _grid()
    q = zero_state(*N3)
    U, a, k = 0.6, 0.3, 1
    q[3] = U
    q[6] = a * np.sin(k * X)
    r = O.rhs(p, q)
    np.testing.assert_allclose(r[4], U * a * k1_mod(k, h[0]) * np.cos(k * X), atol=1e-12)
    assert np.abs(r[5]).max() < 1e-13
    np.testing.assert_allclose(r[6], -eta * a * k2sq_mod(k, h[0]) * np.sin(k * X), atol=1e-12)


@pytest.mark.parametrize("c,d", [(c, d) for c in range(3) for d in range(3) if c != d])
def test_rhs_every_b_component_through_induction(c, d):
    """A = a sin(k x_d) e_c gives B = a k1 cos(k x_d) (e_d x e_c); with a
    uniform u and eta = 0 the induction right-hand side is exactly u x B."""
    p = _p()
    XYZ, h = _grid()
    q = zero_state(*N3)
    a, k = 0.4, 2
    u = np.array([0.3, -0.5, 0.7])
    q[1:4] = u[:, None, None, None]
    q[4 + c] = a * np.sin(k * XYZ[d])
    r = O.rhs(p, q)
    ed, ec = np.eye(3)[d], np.eye(3)[c]
    bdir = np.cross(ed, ec)
    amp = a * k1_mod(k, h[d]) * np.cos(k * XYZ[d])
    want = np.cross(u, bdir)[:, None, None, None] * amp[None]
    np.testing.assert_allclose(r[4:7], want, atol=1e-12)


def test_rhs_forcing_enters_momentum_only():
    p = _p(f0=0.02, sigma=1.0, kmin=1.0, kmax=2.0, seed=9)
    q = zero_state(*N3)
    F = O.forcing_draw(p, step=3, dt=0.01)
    r = O.rhs(p, q, F)
    f = O.forcing_field(p, F)
    np.testing.assert_array_equal(r[1:4], f)
    assert np.abs(r[[0, 4, 5, 6]]).max() == 0.0


# --------------------------------------------------------------------------
# Exact discrete invariants
# --------------------------------------------------------------------------
def test_div_curl_a_vanishes():
    rng = np.random.default_rng(5)
    p = O.Params(nx=10, ny=8, nz=12)
    q = np.zeros(p.shape)
    q[4:7] = rng.standard_normal((3, 12, 8, 10))
    d = O.diagnostics(p, q)
    h = 2 * math.pi / 12
    assert d["divb_max"] < 1e-13 * d["bmax"] / h


def test_periodic_sums_of_derivatives_vanish():
    """Periodic summation by parts: sum D1 f = sum D2 f = sum Dmix f = 0."""
    rng = np.random.default_rng(6)
    p = O.Params(nx=9, ny=8, nz=7)
    f = rng.standard_normal((7, 8, 9))
    for ax in range(3):
        assert abs(O.d1(p, f, ax).sum()) < 1e-11
        assert abs(O.d2(p, f, ax).sum()) < 1e-10
    assert abs(O.dmix(p, f, 0, 2).sum()) < 1e-10


def test_mass_rhs_sums_to_zero_for_uniform_density():
    """ln rho uniform: d ln rho/dt = -div u sums to zero over the grid, so
    the total mass is stationary."""
    rng = np.random.default_rng(7)
    p = O.Params(nx=8, ny=8, nz=8, nu=0.01, eta=0.01)
    q = np.zeros(p.shape)
    q[0] = 0.3
    q[1:4] = 0.1 * rng.standard_normal((3, 8, 8, 8))
    r = O.rhs(p, q)
    assert abs(r[0].sum()) < 1e-12 * np.abs(r[0]).sum()


def test_mass_constant_without_flow():
    """u = 0, A = 0, uniform ln rho: the state is stationary, mass exact."""
    p = O.Params(nx=8, ny=8, nz=8, dt_fixed=0.01, nu=0.0)
    q = np.zeros(p.shape)
    q[0] = 0.25
    m0 = O.diagnostics(p, q)["mass"]
    O.run(p, q, 5)
    assert O.diagnostics(p, q)["mass"] == pytest.approx(m0, rel=1e-15)


# --------------------------------------------------------------------------
# Upwinding of the continuity equation (Sec. 4; reading: fifth-order
# upwind-biased first derivative)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("direction", [1, -1])
@pytest.mark.parametrize("p", range(0, 8))
def test_upwind_stencil_polynomial_exactness(direction, p):
    h, x0 = 0.1, 0.29
    line = [(x0 + s * h) ** p for s in range(-3, 4)]
    exact = p * x0 ** (p - 1) if p > 0 else 0.0
    got = O.stencil_up(line, h, direction)
    if p <= 5:
        assert got == pytest.approx(exact, rel=1e-10, abs=1e-10)
    else:  # order exactly 5
        assert abs(got - exact) > 1e-8


@pytest.mark.parametrize("direction", [1, -1])
def test_upwind_stencil_ignores_the_far_downstream_point(direction):
    """Flow towards +axis: the point three downstream (+3) is not used, the
    point three upstream (-3) is; mirrored for the other direction."""
    rng = np.random.default_rng(11)
    line = rng.standard_normal(7)
    base = O.stencil_up(line, 0.2, direction)
    far_down, far_up = (6, 0) if direction > 0 else (0, 6)
    bumped = line.copy()
    bumped[far_down] += 1.0
    assert O.stencil_up(bumped, 0.2, direction) == base
    bumped = line.copy()
    bumped[far_up] += 1.0
    assert O.stencil_up(bumped, 0.2, direction) != base


def test_upwind_stencil_mirror_symmetry():
    rng = np.random.default_rng(12)
    line = rng.standard_normal(7)
    assert O.stencil_up(line, 0.3, -1) == pytest.approx(-O.stencil_up(line[::-1], 0.3, 1), rel=1e-14)


@pytest.mark.parametrize("U", [0.7, -0.4])
def test_upwinded_advection_of_a_sine_mode(U):
    """ln rho = eps sin(k x), uniform u_x = U: the upwind-biased derivative of
    a Fourier mode is the central one plus a damping part, so
    d ln rho/dt = -U eps k1 cos(kx) - |U| eps (16/(15h)) sin^6(kh/2) sin(kx)
    (the sixth difference of e^{ikx} is -64 sin^6(kh/2) e^{ikx})."""
    n, k, eps = 16, 3, 0.01
    h = 2 * math.pi / n
    X, Y, Z = coords(n, n, n)
    q = zero_state(n, n, n)
    q[0] = eps * np.sin(k * X)
    q[1] = U
    p = O.Params(nx=n, ny=n, nz=n, nu=0.0, eta=0.0, upwind=1)
    r = O.rhs(p, q)
    damp = 16.0 / (15.0 * h) * math.sin(k * h / 2) ** 6
    exact = -U * eps * k1_mod(k, h) * np.cos(k * X) - abs(U) * eps * damp * np.sin(k * X)
    assert np.abs(r[0] - exact).max() < 1e-14
    p0 = O.Params(nx=n, ny=n, nz=n, nu=0.0, eta=0.0, upwind=0)
    r0 = O.rhs(p0, q)
    assert np.abs(r0[0] + U * eps * k1_mod(k, h) * np.cos(k * X)).max() < 1e-14
    # upwinding touches only the continuity equation
    assert np.array_equal(r[1:], r0[1:])


def test_upwinding_in_every_axis():
    """The same closed form along y and z with the flow along that axis."""
    n, k, eps, U = 12, 2, 0.02, 0.5
    h = 2 * math.pi / n
    X, Y, Z = coords(n, n, n)
    damp = 16.0 / (15.0 * h) * math.sin(k * h / 2) ** 6
    for axis, coord in ((1, Y), (2, Z)):
        q = zero_state(n, n, n)
        q[0] = eps * np.sin(k * coord)
        q[1 + axis] = -U
        r = O.rhs(O.Params(nx=n, ny=n, nz=n, nu=0.0, eta=0.0, upwind=1), q)
        exact = U * eps * k1_mod(k, h) * np.cos(k * coord) - U * eps * damp * np.sin(k * coord)
        assert np.abs(r[0] - exact).max() < 1e-14


def _mass_rate(n, mixed):
    """(d/dt sum rho) / sum rho of the semi-discrete continuity equation for a
    smooth periodic state; the continuum value is the integral of
    -div(rho u), i.e. zero."""
    p = O.Params(nx=n, ny=n, nz=n, nu=0.0, eta=0.0)
    X, Y, Z = coords(n, n, n)
    q = np.zeros(p.shape)
    q[0] = 0.3 * np.sin(X + 0.4) * np.cos(Y + Z + 0.2) + 0.2 * np.sin(Z - X + 0.3)
    q[1] = 0.4 * np.sin(X + 2 * Y + 0.1) * np.cos(Z - 0.7)
    q[2] = 0.3 * np.cos(X - 0.5) * np.sin(Y + Z + 0.2)
    q[3] = 0.2 * np.sin(X + Y - Z + 0.9)
    if mixed:  # modes whose wavenumber along a differentiated axis is 2
        q[0] += 0.2 * np.sin(2 * Z - X + 0.3) + 0.1 * np.cos(2 * X + Y)
        q[1] += 0.1 * np.cos(2 * X - Z + 0.5)
        q[2] += 0.1 * np.sin(2 * Y + X)
        q[3] += 0.1 * np.cos(2 * Z + 0.1)
    rho = np.exp(q[0])
    return (rho * O.rhs(p, q)[0]).sum() / rho.sum()


def test_mass_rate_exact_when_every_derivative_sees_one_wavenumber():
    """Every differentiated field has wavenumber 0 or +-1 along the axis of
    its derivative, so D1 = c d/dx exactly with one factor c = k1(1) for
    all three axes; the discrete rate is then c times the trapezoid sum of
    -div(rho u), which vanishes to rounding for a smooth periodic field."""
    for n in (12, 24):
        assert abs(_mass_rate(n, mixed=False)) < 1e-15


def test_mass_drift_converges_at_sixth_order():
    """A ln rho scheme does not conserve sum rho exactly; the rate of mass
    change is the truncation error of D1 (6th order), so it falls by 2^6
    when the grid is refined by 2."""
    r16, r32, r64 = (_mass_rate(n, mixed=True) for n in (16, 32, 64))
    assert abs(r16) > 1e-8  # not zero: the test sees the truncation error
    for a, b in ((r16, r32), (r32, r64)):
        order = math.log2(abs(a / b))
        assert 5.6 < order < 6.3, order


# --------------------------------------------------------------------------
# Time integration: exact linear decays at the modified wavenumber
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nsteps", [1, 7])
def test_beltrami_resistive_decay(nsteps):
    n, k, eta, dt = 16, 2, 0.05, 0.03
    p = O.Params(nx=n, ny=n, nz=n, eta=eta, nu=0.02, dt_fixed=dt)
    X, Y, Z = coords(n, n, n)
    q = zero_state(n)
    q[4] = np.sin(k * Z)
    q[5] = np.cos(k * Z)
    O.run(p, q, nsteps)
    h = 2 * math.pi / n
    g = rk3_gain(-eta * k2sq_mod(k, h) * dt) ** nsteps
    np.testing.assert_allclose(q[4], g * np.sin(k * Z), atol=1e-13)
    np.testing.assert_allclose(q[5], g * np.cos(k * Z), atol=1e-13)
    assert np.abs(q[:4]).max() < 1e-13 and np.abs(q[6]).max() < 1e-13


@pytest.mark.parametrize("U", [0.1, 0.9])
def test_shear_wave_viscous_decay(U):
    n, k, nu, dt, ns = 12, 1, 0.07, 0.05, 5
    p = O.Params(nx=n, ny=n, nz=n, nu=nu, eta=0.0, dt_fixed=dt)
    X, Y, Z = coords(n, n, n)
    q = zero_state(n)
    q[1] = U * np.sin(k * Z)
    O.run(p, q, ns)
    g = rk3_gain(-nu * k2sq_mod(k, 2 * math.pi / n) * dt) ** ns
    np.testing.assert_allclose(q[1], g * U * np.sin(k * Z), atol=1e-13)
    assert np.abs(q[[0, 2, 3, 4, 5, 6]]).max() < 1e-13


def test_third_order_time_convergence():
    """Smooth nonlinear state, fixed final time: the Richardson ratio of
    successive dt halvings approaches 2^3."""
    from paper_2012_08758_b300.inputs import random_modes_state
    n, T = 8, 0.24
    sols = []
    for m in (6, 12, 24):
        p = O.Params(nx=n, ny=n, nz=n, nu=0.02, eta=0.02, dt_fixed=T / m)
        q = random_modes_state(n, seed=11, amp=0.2, kmax=1, nmodes=3)
        O.run(p, q, m)
        sols.append(q)
    ratio = np.abs(sols[0] - sols[1]).max() / np.abs(sols[1] - sols[2]).max()
    assert 7.0 < ratio < 9.0, ratio


# --------------------------------------------------------------------------
# Forcing (Eqs. 4-6)
# --------------------------------------------------------------------------
def test_kshell_counts_and_bounds():
    sh = O.kshell(2.5, 3.5)
    assert len(sh) == 98
    m = np.linalg.norm(sh, axis=1)
    assert m.min() >= 2.5 and m.max() <= 3.5
    assert len(O.kshell(4.5, 5.5)) == 350


@pytest.mark.parametrize("kmin,kmax", [(1.0, 2.0), (3.0, 3.0), (2.0, 3.0), (4.5, 5.5)])
def test_kshell_bounds_are_inclusive(kmin, kmax):
    want = sorted((a, b, c) for a in range(-6, 7) for b in range(-6, 7) for c in range(-6, 7)
                  if kmin * kmin <= a * a + b * b + c * c <= kmax * kmax)
    assert sorted(map(tuple, O.kshell(kmin, kmax).tolist())) == want


def test_splitmix64_published_vector():
    path = os.path.join(GOLDEN, "splitmix64_seed1234567.txt")
    vals = [int(l.split()[0]) for l in open(path) if l.strip() and not l.startswith("#")]
    assert [O.splitmix64(1234567, i) for i in range(len(vals))] == vals


@pytest.mark.parametrize("sigma", [0.0, 0.5, 1.0])
def test_forcing_eigenfunction_properties(sigma):
    p = O.Params(nx=16, ny=16, nz=16, sigma=sigma, f0=0.02, kmin=2.5, kmax=3.5, seed=4)
    for step in range(20):
        F = O.forcing_draw(p, step)
        a, b, kp = map(np.array, (F.a, F.b, F.kp))
        assert np.dot(a, a) + np.dot(b, b) == pytest.approx(1.0, rel=1e-14)
        assert abs(np.dot(kp, a)) < 1e-14 and abs(np.dot(kp, b)) < 1e-14
        assert np.dot(a, a) == pytest.approx(1.0 / (1.0 + sigma ** 2), rel=1e-14)
        # helicity <f . curl f> / (|k| <f^2>) = -2 a.(k x b)/|k| = 2 sigma/(1+sigma^2)
        hel = -2.0 * np.dot(a, np.cross(kp, b)) / np.linalg.norm(kp)
        assert hel == pytest.approx(2 * sigma / (1 + sigma ** 2), abs=1e-14)
        assert -math.pi <= F.phi < math.pi
        assert np.linalg.norm(F.e) == pytest.approx(1.0, rel=1e-15)
        assert abs(np.dot(kp, F.e)) <= 0.99 * np.linalg.norm(kp)


def test_forcing_field_is_a_single_fourier_mode():
    """f = Re{N f_k e^{i(k.x+phi)}}: the FFT has only the modes +-k, with
    amplitude N^3 * N f_k e^{i phi} / 2 at +k; <f^2> = N_amp^2 / 2."""
    n = 12
    p = O.Params(nx=n, ny=n, nz=n, sigma=0.7, f0=0.05, kmin=2.5, kmax=3.5, seed=12)
    F = O.forcing_draw(p, step=5, dt=0.02)
    f = O.forcing_field(p, F)
    amp = F.amp
    assert amp == pytest.approx(0.05 * 1.0 * math.sqrt(np.linalg.norm(F.kp) / 0.02), rel=1e-15)
    assert np.mean(f ** 2) * 3 == pytest.approx(amp ** 2 / 2, rel=1e-12)
    fk = np.array(F.a) + 1j * np.array(F.b)
    kx, ky, kz = F.k
    for d in range(3):
        spec = np.fft.fftn(f[d])  # axes (z, y, x)
        want = n ** 3 * amp * fk[d] * np.exp(1j * F.phi) / 2
        assert abs(spec[kz % n, ky % n, kx % n] - want) < 1e-10
        spec[kz % n, ky % n, kx % n] = 0
        spec[-kz % n, -ky % n, -kx % n] = 0
        assert np.abs(spec).max() < 1e-10


def test_forcing_once_per_step_adds_dt_f_to_u():
    """Forcing mode 1 (the alternative reading of where the forcing enters
    the RK step): a gas at rest with uniform density, A = 0 and no diffusion
    has a zero right-hand side without forcing, so one step leaves ln rho and
    A as they were and sets u to dt * f(x) -- once, with the step's own dt in
    the normalisation of Eq. 5 and the draw of that step index."""
    nx, ny, nz, dt = 12, 10, 8, 0.013
    p = O.Params(nx=nx, ny=ny, nz=nz, nu=0.0, eta=0.0, f0=0.05, sigma=0.7, kmin=2.5, kmax=3.5,
                 seed=5, dt_fixed=dt, forcing_mode=1)
    q = zero_state(nx, ny, nz)
    q[0] = 0.3
    d, F = O.step(p, q, step_index=4)
    assert d == dt
    G = O.forcing_draw(p, 4, dt=dt)
    assert F.k == G.k and F.amp == G.amp
    f = O.forcing_field(p, G)
    np.testing.assert_allclose(q[1:4], dt * f, rtol=0, atol=1e-16)
    assert np.abs(q[1:4]).max() > 1e-4  # the forcing is really there
    assert np.all(q[0] == 0.3) and np.all(q[4:] == 0.0)


def test_forcing_once_per_step_is_the_unforced_step_plus_dt_f():
    """On a general state, forcing mode 1 equals the unforced RK3 step (same
    dt) followed by u += dt * f of the step's draw; mode 0 differs from it
    only at second order in dt (RK3 applies a constant forcing with total
    weight dt over the three substeps)."""
    from paper_2012_08758_b300.inputs import random_modes_state
    n, dt = 10, 0.004
    base = dict(nx=n, ny=n, nz=n, nu=0.02, eta=0.03, f0=0.05, sigma=0.4, seed=9, dt_fixed=dt)
    q0 = random_modes_state(n, seed=3, amp=0.2, kmax=2, nmodes=4)
    q1 = q0.copy()
    O.step(O.Params(**base, forcing_mode=1), q1, step_index=2)
    qu = q0.copy()
    O.step(O.Params(**dict(base, f0=0.0)), qu, step_index=2)
    f = O.forcing_field(O.Params(**base), O.forcing_draw(O.Params(**base), 2, dt=dt))
    np.testing.assert_allclose(q1[[0, 4, 5, 6]], qu[[0, 4, 5, 6]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(q1[1:4], qu[1:4] + dt * f, rtol=0, atol=1e-15)
    q0m = q0.copy()
    O.step(O.Params(**base, forcing_mode=0), q0m, step_index=2)
    diff = np.abs(q0m - q1).max()
    assert 0 < diff < 20 * dt * dt * np.abs(f).max()


def test_forcing_draw_covers_shell_uniformly():
    p = O.Params(f0=0.02, kmin=2.5, kmax=3.5, seed=77)
    sh = {tuple(v) for v in O.kshell(2.5, 3.5)}
    seen = {}
    phis, es = [], []
    for s in range(3000):
        F = O.forcing_draw(p, s)
        seen[F.k] = seen.get(F.k, 0) + 1
        phis.append(F.phi)
        es.append(F.e)
    assert set(seen) <= sh and len(seen) == len(sh)
    assert abs(np.mean(phis)) < 0.12
    assert np.abs(np.mean(es, axis=0)).max() < 0.05


# --------------------------------------------------------------------------
# Time step, diagnostics, growth-rate fit
# --------------------------------------------------------------------------
def test_dt_rule_closed_forms():
    n = 8
    p = O.Params(nx=n, ny=n, nz=n, cs=1.5, nu=1e-3, eta=2e-3, cfl=0.4, cfl_visc=0.08)
    q = zero_state(n)
    q[1], q[2] = 0.3, 0.4  # |u| = 0.5
    h = 2 * math.pi / n
    assert O.dt(p, q) == pytest.approx(0.4 * h / (0.5 + 1.5), rel=1e-15)
    p.nu, p.eta = 5.0, 1.0  # diffusive limit binds
    assert O.dt(p, q) == pytest.approx(0.08 * h * h / 5.0, rel=1e-15)
    p.dt_fixed = 1.19209e-7
    assert O.dt(p, q) == 1.19209e-7


def test_dt_uses_smallest_spacing():
    p = O.Params(nx=8, ny=16, nz=12, cs=1.0, nu=0.0, eta=0.0, cfl=0.4)
    q = zero_state(8, 16, 12)
    assert O.dt(p, q) == pytest.approx(0.4 * (2 * math.pi / 16) / 1.0, rel=1e-15)


def test_dt_includes_fast_magnetosonic_speed():
    """A = (sin kz, cos kz, 0): |B| = k1 everywhere, so
    v = sqrt(cs^2 + k1^2 / rho)."""
    n, k, c = 12, 1, 0.5
    p = O.Params(nx=n, ny=n, nz=n, nu=0.0, eta=0.0)
    X, Y, Z = coords(n, n, n)
    q = zero_state(n)
    q[0] = c
    q[4], q[5] = np.sin(k * Z), np.cos(k * Z)
    k1 = k1_mod(k, 2 * math.pi / n)
    assert O.max_speed(p, q) == pytest.approx(math.sqrt(1 + k1 * k1 / math.exp(c)), rel=1e-14)


def test_diagnostics_closed_forms():
    n, k = 12, 2
    p = O.Params(nx=n, ny=n, nz=n)
    X, Y, Z = coords(n, n, n)
    q = zero_state(n)
    c, U = 0.3, 0.8
    q[0] = c
    q[1] = U * np.sin(k * Y)
    q[4], q[5] = np.sin(k * Z), np.cos(k * Z)
    d = O.diagnostics(p, q)
    k1 = k1_mod(k, 2 * math.pi / n)
    assert d["urms"] == pytest.approx(U / math.sqrt(2), rel=1e-14)
    assert d["umax"] == pytest.approx(U * np.abs(np.sin(k * Y)).max(), rel=1e-15)
    assert d["brms"] == pytest.approx(k1, rel=1e-14)
    assert d["bmax"] == pytest.approx(k1, rel=1e-14)
    assert d["emag"] == pytest.approx(k1 * k1 / 2, rel=1e-14)
    assert d["ekin"] == pytest.approx(math.exp(c) * U * U / 4, rel=1e-14)
    assert d["mass"] == pytest.approx(math.exp(c), rel=1e-15)


def test_growth_rate_fit_recovers_exponential():
    t = np.linspace(0, 50, 101)
    assert O.growth_rate(t, 1e-5 * np.exp(0.0173 * t)) == pytest.approx(0.0173, rel=1e-12)


# --------------------------------------------------------------------------
# Magnetic energy spectrum (Sec. 5, power spectra)
# --------------------------------------------------------------------------
def test_spectrum_of_one_mode_sits_in_its_shell():
    """A_z = sin(3x + 0.2): B_y = -k1(3) cos(3x + 0.2) exactly, so all of
    <B^2>/2 = k1^2/4 lies in shell 3."""
    n = 16
    h = 2 * math.pi / n
    X, Y, Z = coords(n, n, n)
    q = zero_state(n)
    q[6] = np.sin(3 * X + 0.2)
    p = O.Params(nx=n, ny=n, nz=n)
    E = O.spectrum(p, q)
    assert len(E) == 15  # floor(sqrt(3 * 8^2) + 1/2) + 1
    want = k1_mod(3, h) ** 2 / 4
    assert E[3] == pytest.approx(want, rel=1e-13)
    assert np.abs(np.delete(E, 3)).max() < 1e-15 * want


def test_spectrum_of_a_diagonal_mode():
    """A_z = sin(3x + 4y): |k| = 5; B_x = k1(4) cos, B_y = -k1(3) cos."""
    n = 20
    h = 2 * math.pi / n
    X, Y, Z = coords(n, n, n)
    q = zero_state(n)
    q[6] = np.sin(3 * X + 4 * Y)
    E = O.spectrum(O.Params(nx=n, ny=n, nz=n), q)
    want = (k1_mod(3, h) ** 2 + k1_mod(4, h) ** 2) / 4
    assert E[5] == pytest.approx(want, rel=1e-13)
    assert np.abs(np.delete(E, 5)).max() < 1e-15 * want


@pytest.mark.parametrize("k,shell", [((1, 1, 0), 1), ((1, 1, 1), 2), ((2, 1, 1), 2), ((2, 2, 1), 3),
                                     ((3, 2, 0), 4), ((4, 4, 2), 6)])
def test_spectrum_shell_is_the_nearest_integer_of_k(k, shell):
    """Shell m holds m - 1/2 <= |k| < m + 1/2: sqrt2 -> 1, sqrt3 -> 2,
    sqrt6 -> 2, 3 -> 3, sqrt13 -> 4, 6 -> 6."""
    n = 12
    X, Y, Z = coords(n, n, n)
    q = zero_state(n)
    q[4] = np.cos(k[0] * Y + k[1] * Z + k[2] * X + 0.4)  # A_x varying in y, z (and x)
    E = O.spectrum(O.Params(nx=n, ny=n, nz=n), q)
    assert E[shell] > 0
    assert np.abs(np.delete(E, shell)).max() < 1e-14 * E[shell]


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 10, 8), (9, 7, 5)])
def test_spectrum_sums_to_the_magnetic_energy(shape):
    """Parseval: sum_m E_B(m) = <B^2>/2, the real-space mean of the
    diagnostics (compensated sum); shell 0 (mean field) vanishes."""
    nx, ny, nz = shape
    rng = np.random.default_rng(9)
    p = O.Params(nx=nx, ny=ny, nz=nz)
    q = 0.1 * rng.standard_normal(p.shape)
    E = O.spectrum(p, q)
    m = int(math.floor(math.sqrt((nx // 2) ** 2 + (ny // 2) ** 2 + (nz // 2) ** 2) + 0.5))
    assert len(E) == m + 1
    assert E.sum() == pytest.approx(O.diagnostics(p, q)["emag"], rel=1e-13)
    assert E[0] < 1e-28 * E.sum()


def test_channel_growth_rates_of_exact_exponentials():
    from paper_2012_08758_b300.growth import channel_growth_rates
    t = np.linspace(0.0, 3.0, 13)
    lam = np.array([0.0, 0.3, -0.1, 0.05])
    S = np.exp(2 * lam[None, :] * t[:, None]) * np.array([1.0, 2e-3, 5.0, 1e-8])
    got = channel_growth_rates(t, S, channels=[1, 2, 3])
    for k in (1, 2, 3):
        assert got[k] == pytest.approx(lam[k], rel=1e-12, abs=1e-13)


def test_golden_tables_of_growth_rates_are_complete():
    """The stored Tables 1-2 (25 helical, 27 non-helical rows): helical
    growth rates are all positive; non-helical ones change sign between
    Re_M 17 and 28 (the small-scale dynamo onset the paper reports)."""
    rows = [line.split() for line in open(os.path.join(GOLDEN, "growth_rates_tables_1_2.txt"))
            if line.strip() and not line.startswith("#")]
    hel = [r for r in rows if r[0] == "1"]
    non = [r for r in rows if r[0] == "0"]
    assert len(hel) == 25 and len(non) == 27
    assert all(float(r[3]) > 0 for r in hel)
    for r in non:
        assert (float(r[3]) > 0) == (float(r[4]) > 25.0)
