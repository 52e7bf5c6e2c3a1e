"""Closed-form test states and the closed-form responses of the discrete
operators to them (plain numpy)."""
import math

import numpy as np


def coords(nx, ny, nz, lx=2 * math.pi, ly=2 * math.pi, lz=2 * math.pi):
    x = np.arange(nx) * (lx / nx)
    y = np.arange(ny) * (ly / ny)
    z = np.arange(nz) * (lz / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def k1_mod(k, h):
    """Modified wavenumber of the 6th-order first-derivative stencil on
    sin(k x): k1 h = (45 sin t - 9 sin 2t + sin 3t) / 30, t = k h."""
    t = k * h
    return (45 * math.sin(t) - 9 * math.sin(2 * t) + math.sin(3 * t)) / (30 * h)


def k2sq_mod(k, h):
    """Modified squared wavenumber of the 6th-order second-derivative
    stencil: k2^2 h^2 = (490 - 540 cos t + 54 cos 2t - 4 cos 3t) / 180."""
    t = k * h
    return (490 - 540 * math.cos(t) + 54 * math.cos(2 * t) - 4 * math.cos(3 * t)) / (180 * h * h)


def kmix_mod(k, l, ha, hb):
    """Mixed-stencil factor on sin(k a) sin(l b): the result is
    cos(k a) cos(l b) * kmix (four-term diagonal identity)."""
    t, s = k * ha, l * hb
    return (270 * math.sin(t) * math.sin(s) - 27 * math.sin(2 * t) * math.sin(2 * s)
            + 2 * math.sin(3 * t) * math.sin(3 * s)) / (180 * ha * hb)


def rk3_gain(z):
    """Amplification factor of any 3-stage 3rd-order RK on y' = lambda y."""
    return 1 + z + z * z / 2 + z ** 3 / 6


def zero_state(nx, ny=None, nz=None):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return np.zeros((7, nz, ny, nx))
