"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/mhd.h declares; host-only logic (defaults, validation,
workspace sizing) runs without a GPU.  No kernel is launched here."""
import ctypes as C
import os
import re

import numpy as np

import pytest

from paper_2012_08758_b300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    from paper_2012_08758_b300 import binding
    return binding


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mhd_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mhd_create", "mhd_step", "mhd_reduce", "mhd_destroy", "mhd_set_state",
                 "mhd_get_state", "mhd_batch_create", "mhd_batch_step"):
        assert must in names


def test_library_exports_every_declared_symbol(B):
    L = B.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_uses_the_same_names(B):
    import paper_2012_08758_b300 as pkg
    for n in declared_functions():
        assert hasattr(B, n), n
        assert getattr(pkg, n) is getattr(B, n)


def test_default_params(B):
    p = B.mhd_default_params()
    assert (p.nx, p.ny, p.nz) == (32, 32, 32)
    assert abs(p.lx - 2 * 3.141592653589793) < 1e-15
    assert p.cs == 1.0 and p.nu == 5e-3 and p.eta == 5e-3
    assert p.cfl == 0.4 and p.dtype == B.MHD_F32 and p.f0 == 0.0


def test_workspace_bytes_scale_with_grid(B):
    small = B.mhd_workspace_bytes(B.mhd_default_params(nx=32, ny=32, nz=32))
    big = B.mhd_workspace_bytes(B.mhd_default_params(nx=64, ny=64, nz=64))
    dbl = B.mhd_workspace_bytes(B.mhd_default_params(nx=64, ny=64, nz=64, dtype=B.MHD_F64))
    # 21 padded arrays of (nx+8 rounded to 8) x (ny+6) x (nz+6) values
    assert big >= 21 * 72 * 70 * 70 * 4
    assert 1.9 < dbl / big < 2.01 and big > small


@pytest.mark.parametrize("dtype,tiles", [(0, range(0, 29)), (1, range(0, 5))])
def test_every_tile_variant_is_accepted(B, dtype, tiles):
    """FP32 TMA tiles 1-28 (shapes, stage counts, barrier spacings, packed
    pairs, paired points, w layouts) and FP64 tiles 1-4, and 0 for the
    default, are valid parameters."""
    for t in tiles:
        assert B.mhd_workspace_bytes(B.mhd_default_params(nx=40, ny=24, nz=16, kernel=2, tile=t, dtype=dtype)) > 0


@pytest.mark.parametrize("bad,msg", [
    (dict(nx=0), "nx"), (dict(cs=0.0), "cs"), (dict(nu=-1.0), "nu"),
    (dict(f0=0.1, kmin=0.0), "shell"), (dict(f0=0.1, kmin=0.2, kmax=0.5), "no integer"),
    (dict(f0=0.1, sigma=1.5), "sigma"), (dict(dtype=7), "dtype"), (dict(forcing_mode=3), "forcing_mode"), (dict(upwind=2), "upwind"),
    (dict(cfl=0.0), "cfl"), (dict(kernel=99), "kernel"),
    (dict(kernel=2, tile=29), "tile"), (dict(kernel=2, tile=6, dtype=1), "tile"), (dict(kernel=1, tile=3), "tile"),
])
def test_invalid_parameters_are_rejected(B, bad, msg):
    with pytest.raises(B.MhdError) as e:
        B.mhd_workspace_bytes(B.mhd_default_params(**bad))
    assert e.value.code == B.MHD_EINVAL and msg in str(e.value)


def test_alu_peak_rejects_bad_arguments_without_touching_the_gpu(B):
    """Argument checks of the measurement helper run before any CUDA call."""
    L = B.lib()
    import ctypes as C
    f = C.c_double()
    assert L.mhd_alu_peak(7, None, C.byref(f), None) == B.MHD_EINVAL
    assert L.mhd_alu_peak(B.MHD_F32, None, None, None) == B.MHD_EINVAL


def test_spectrum_shell_count_and_box_checks(B):
    assert B.mhd_spectrum_shells(B.mhd_default_params(nx=16, ny=16, nz=16)) == 15
    assert B.mhd_spectrum_shells(B.mhd_default_params(nx=9, ny=7, nz=5)) == 6  # sqrt(16+9+4)=5.39
    for bad in (dict(lx=1.0), dict(nx=1)):
        with pytest.raises(B.MhdError) as e:
            B.mhd_spectrum_shells(B.mhd_default_params(**bad))
        assert e.value.code == B.MHD_EINVAL


def test_seed_field_rejects_null_context(B):
    import ctypes as C
    assert B.lib().mhd_set_seed_field(None, C.c_uint64(1), C.c_double(1e-5)) == B.MHD_EINVAL


@pytest.mark.parametrize("shape,grid", [((256, 256, 256), 148), ((512, 512, 512), 148), ((64, 64, 64), 148),
                                        ((37, 23, 11), 148), ((1, 1, 1), 148), ((45, 37, 29), 444),
                                        ((256, 96, 40), 296), ((300, 200, 100), 148), ((256, 240, 128), 148)])
@pytest.mark.parametrize("tile", [0, 2, 4, 5, 9, 16, 17, 19, 20, 25, 28])
def test_substep_plan_covers_every_point_once(B, shape, grid, tile):
    """The work split of the fused substep: every (x-y tile, z) of the grid
    exactly once, table rectangular over the CTAs it uses, whole columns
    first, and the per-CTA load balanced when there is enough work."""
    nx, ny, nz = shape
    p = B.mhd_default_params(nx=nx, ny=ny, nz=nz, kernel=B.MHD_KERNEL_TMA, tile=tile)
    tiles, g = B.mhd_substep_plan(p, grid)
    assert 1 <= g <= grid and len(tiles) % g == 0
    # tile 0: the warp-specialised paired-point tile 28 (64 x 8 columns)
    res = B.mhd_resolve_params(p).tile
    assert res == (tile if tile else 28)
    tw = 64 if res >= 17 else 32
    th = {2: 4, 4: 12, 5: 12, 9: 6, 13: 12, 16: 12, 17: 8, 18: 8, 19: 4, 20: 6, 22: 8, 25: 8, 26: 8, 28: 8}[res]
    seen = {}
    for x0, y0, z0, z1, run in tiles:
        assert run == 0
        if z1 <= z0:
            continue
        assert x0 % tw == 0 and y0 % th == 0 and 0 <= z0 < z1 <= nz
        cov = seen.setdefault((x0, y0), np.zeros(nz, dtype=int))
        cov[z0:z1] += 1
    cols = {(x0, y0) for x0 in range(0, nx, tw) for y0 in range(0, ny, th)}
    assert set(seen) == cols
    assert all((c == 1).all() for c in seen.values())
    planes = np.zeros(g)
    for k, (x0, y0, z0, z1, run) in enumerate(tiles):
        planes[k % g] += max(0, z1 - z0)
    # balance in planes is only meaningful without ragged (partly idle) tiles,
    # which the plan weights by their lower cost; faces weigh up to 1.16x
    if nx * ny * nz >= 128 ** 3 and nx % tw == 0 and ny % th == 0:
        assert planes.max() <= 1.15 * planes.mean()


@pytest.mark.parametrize("shape", [(256, 256, 256), (384, 384, 384), (512, 512, 512), (320, 320, 320)])
def test_paired_split_keeps_every_sm_busy(B, shape):
    """Paired kernel: the split uses all 148 CTAs even where one or two
    waves of whole columns would fit (256^3: 128 columns of 64 x 8; 384^3:
    288), cutting columns end to end so that every CTA gets the same load."""
    nx, ny, nz = shape
    p = B.mhd_default_params(nx=nx, ny=ny, nz=nz, kernel=B.MHD_KERNEL_TMA, tile=28)
    tiles, g = B.mhd_substep_plan(p, 148)
    assert g == 148
    planes = np.zeros(g)
    for k, (x0, y0, z0, z1, run) in enumerate(tiles):
        planes[k % g] += max(0, z1 - z0)
    assert planes.min() > 0


@pytest.mark.parametrize("shape", [(256, 256, 256), (384, 384, 384), (512, 512, 512), (1024, 1024, 256), (33, 17, 9)])
def test_default_tile_choice(B, shape):
    """Automatic kernel and tile: FP32 takes the paired-point kernel with w
    interleaved (tile 28), FP64 tile 3; an explicit tile is kept."""
    nx, ny, nz = shape
    r = B.mhd_resolve_params(B.mhd_default_params(nx=nx, ny=ny, nz=nz))
    assert (r.kernel, r.tile) == (B.MHD_KERNEL_TMA, 28)
    r = B.mhd_resolve_params(B.mhd_default_params(nx=nx, ny=ny, nz=nz, dtype=B.MHD_F64))
    assert (r.kernel, r.tile) == (B.MHD_KERNEL_TMA, 3)
    r = B.mhd_resolve_params(B.mhd_default_params(nx=nx, ny=ny, nz=nz, kernel=B.MHD_KERNEL_TMA, tile=26))
    assert r.tile == 26
    r = B.mhd_resolve_params(B.mhd_default_params(nx=nx, ny=ny, nz=nz, kernel=B.MHD_KERNEL_SMEM))
    assert (r.kernel, r.tile) == (B.MHD_KERNEL_SMEM, 0)
    with pytest.raises(B.MhdError):
        B.mhd_resolve_params(B.mhd_default_params(nx=0))


def test_autotuner_candidates_cover_every_accepted_variant(B):
    """The autotuner tries every (kernel, tile) the library accepts for each
    dtype and nothing it rejects: all TMA tiles up to the first invalid id,
    and the plane-ring kernel."""
    from paper_2012_08758_b300 import autotune
    for dtype in (B.MHD_F32, B.MHD_F64):
        valid = []
        t = 1
        while True:
            try:
                B.mhd_workspace_bytes(B.mhd_default_params(kernel=B.MHD_KERNEL_TMA, tile=t, dtype=dtype))
            except B.MhdError:
                break
            valid.append((B.MHD_KERNEL_TMA, t))
            t += 1
        assert sorted(autotune.CANDIDATES[dtype]) == sorted(valid + [(B.MHD_KERNEL_SMEM, 0)])


def test_padding_check_rejects_null(B):
    import ctypes as C
    n = C.c_longlong()
    assert B.lib().mhd_padding_check(None, C.byref(n)) == B.MHD_EINVAL
