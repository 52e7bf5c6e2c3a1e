"""Mutation check of the oracle's pins: each case plants one plausible
mistake (a dropped factor, a wrong sign, a transposed operand, a wrong
index) in a scratch copy of the oracle's C source (built with gcc in a
temporary folder) or of its Python side, and runs the pin suite against it;
every mutant must fail.  CPU only; the committed oracle is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mhd_oracle.c")

MUTANTS = {
    "lorentz_sign": ("JxB[a] / rho", "-JxB[a] / rho"),
    "grad_div_third": ("gdu[a] / 3.0", "gdu[a] / 2.0"),
    "strain_factor_two": ("2.0 * Sg", "1.0 * Sg"),
    "strain_trace": ("divu / 3.0 : 0.0", "divu / 2.0 : 0.0"),
    "u_cross_b_order": ("cross3(uu, B, uxB);", "cross3(B, uu, uxB);"),
    "bz_sign": ("gA[1][0] - gA[0][1]};\n  /* Lap", "gA[0][1] - gA[1][0]};\n  /* Lap"),
    "bx_sign": ("/* B = curl A */\n  double B[3] = {gA[2][1] - gA[1][2],",
                "/* B = curl A */\n  double B[3] = {gA[1][2] - gA[2][1],"),
    "d1_weight": ("- 9.0 * (f[2] - f[-2])", "- 8.0 * (f[2] - f[-2])"),
    "d2_weight": ("- 27.0 * (f[2] + f[-2])", "- 26.0 * (f[2] + f[-2])"),
    "dmix_weight": ("- 27.0 * S[2]", "- 26.0 * S[2]"),
    "dmix_pattern": ("P(s, s) + P(-s, -s) - P(s, -s) - P(-s, s)",
                     "P(s, s) - P(-s, -s) + P(s, -s) - P(-s, s)"),
    "dmix_axis": ("offset(b, sb, &bi, &bj, &bk);", "offset(a, sb, &bi, &bj, &bk);"),
    "rk_alpha": ("-153.0 / 128.0", "-150.0 / 128.0"),
    "rk_beta": ("15.0 / 16.0, 8.0", "14.0 / 16.0, 8.0"),
    "advection_transposed": ("uu[0] * G[a][0] + uu[1] * G[a][1]", "uu[0] * G[0][a] + uu[1] * G[1][a]"),
    "pressure_cs_not_squared": ("- cs2 * g[a]", "- p->cs * g[a]"),
    "continuity_div_sign": ("- divu;\n", "+ divu;\n"),
    "eta_vs_nu": ("p->eta * lapA[a]", "p->nu * lapA[a]"),
    "helicity_sign": ("F->b[d] = -p->sigma", "F->b[d] = p->sigma"),
    "forcing_norm_dt": ("sqrt(kk * p->cs / dt)", "sqrt(kk * p->cs * dt)"),
    "forcing_phase_sign": ("+ F->phi;", "- F->phi;"),
    "forcing_sin_sign": ("F->a[d] * c - F->b[d] * s", "F->a[d] * c + F->b[d] * s"),
    "shell_exclusive": ("m >= kmin && m <= kmax", "m > kmin && m <= kmax"),
    "dt_max_spacing": ("double dmin = fmin(spacing(p, 0),", "double dmin = fmax(spacing(p, 0),"),
    "dt_alfven_rho": ("sqrt(cs2 + B2 / exp(q[c]))", "sqrt(cs2 + B2 * exp(q[c]))"),
    "ekin_density": ("kadd(&sk, rho * u2);", "kadd(&sk, u2);"),
    "upwind_downstream": ("uu[a] >= 0.0 ? 1 : -1", "uu[a] >= 0.0 ? -1 : 1"),
    "upwind_weight": ("+ 30.0 * f[1] - 3.0 * f[2]", "+ 30.0 * f[1] - 2.0 * f[2]"),
    "upwind_ignored": ("p->upwind ? orc_dup", "0 ? orc_dup"),
    "mode1_third_dt": ("q[(1 + a) * n + c] += dt * f[a];", "q[(1 + a) * n + c] += dt / 3.0 * f[a];"),
    "mode1_into_A": ("q[(1 + a) * n + c] += dt * f[a];", "q[(4 + a) * n + c] += dt * f[a];"),
    "mode1_sign": ("q[(1 + a) * n + c] += dt * f[a];", "q[(1 + a) * n + c] -= dt * f[a];"),
    "mode1_also_in_rhs": ("p->forcing_mode == 0) orc_forcing_at", "p->forcing_mode >= 0) orc_forcing_at"),
}


def _run_pins_with_c_source(tmp_path, src):
    """Pins against a scratch build of the C source `src`, compiled with the
    oracle's own flags and loaded through ORACLE_LIB_OVERRIDE."""
    from oracle import oracle as O
    mut = tmp_path / "mutant.c"
    mut.write_text(src)
    lib = O.compile_oracle(str(mut), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=lib)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                          env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)


def test_c_mutation_harness_passes_the_unmodified_oracle(tmp_path):
    """Control: the unmodified source through the same scratch build and
    library override passes every pin, so a failing mutant fails for its
    planted mistake and not for the harness."""
    r = _run_pins_with_c_source(tmp_path, open(SRC).read())
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation site not unique/found: {name}"
    r = _run_pins_with_c_source(tmp_path, src.replace(before, after))
    assert r.returncode != 0, f"mutant {name} survived the pins"


# Mistakes planted in the Python side of the oracle (the spectrum's shells
# and normalisation, the growth-rate fit), run against the same pins with
# the committed C library.
PY_SRC = os.path.join(ROOT, "oracle", "oracle.py")
PY_MUTANTS = {
    "shell_floor_not_nearest": ("np.floor(np.sqrt(K2) + 0.5)", "np.floor(np.sqrt(K2))"),
    "spectrum_half_dropped": ("return 0.5 * np.bincount", "return 1.0 * np.bincount"),
    "spectrum_norm_once": ("/ float(n) ** 2", "/ float(n)"),
    "spectrum_drops_kx": (" + kx[None, None, :] ** 2", ""),
    "growth_fit_intercept": ("np.polyfit(t, y, 1)[0]", "np.polyfit(t, y, 1)[1]"),
    "growth_fit_no_log": ("y = np.log(np.asarray(brms, dtype=np.float64))",
                          "y = np.asarray(brms, dtype=np.float64)"),
}


def _run_pins_with_python_oracle(tmp_path, src):
    """Pins against a scratch package `oracle` whose oracle.py is `src`
    (the committed C library loaded through ORACLE_LIB_OVERRIDE)."""
    from oracle import oracle as O
    lib = O.build()
    import shutil
    pkg = tmp_path / "root"
    (pkg / "oracle").mkdir(parents=True)
    (pkg / "oracle" / "__init__.py").write_text("")
    (pkg / "oracle" / "oracle.py").write_text(src)
    # the pins and their helpers, copied so that their root (put first on
    # sys.path by the copied conftest) is the scratch one
    tests = pkg / "tests"
    tests.mkdir()
    for f in ("__init__.py", "conftest.py", "states.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tests / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tests / "golden")
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=lib,
               PYTHONPATH=os.pathsep.join([str(pkg), ROOT, os.environ.get("PYTHONPATH", "")]))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           str(tests / "test_oracle_pins.py")],
                          env=env, cwd=str(pkg), capture_output=True, text=True, timeout=600)


def test_python_mutation_harness_passes_the_unmodified_oracle(tmp_path):
    """Control: the harness itself (scratch package, library override) lets
    the committed oracle pass, so a failing mutant fails for its mistake."""
    r = _run_pins_with_python_oracle(tmp_path, open(PY_SRC).read())
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pins_reject_python_mutant(name, tmp_path):
    before, after = PY_MUTANTS[name]
    src = open(PY_SRC).read()
    assert src.count(before) == 1, f"mutation site not unique/found: {name}"
    r = _run_pins_with_python_oracle(tmp_path, src.replace(before, after))
    assert r.returncode != 0, f"mutant {name} survived the pins"
