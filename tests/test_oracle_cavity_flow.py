"""Pin of the walled cavity with flow, corners included.

With porosity -> 1, Da -> infinity, F_phi = 0, H_v = 0 and a PCM that stays
liquid, the Sec. IV B cavity becomes the differentially heated square cavity
of natural convection, whose steady mean hot-wall Nusselt number is a
published benchmark (``tests/golden/de_vahl_davis_1983.json``).  Every wall
node here goes through Eq. 52 (non-equilibrium extrapolation from the inward
neighbour, diagonal at corners), so the pin covers the wall rule with flow,
the buoyancy force (Eq. 7), the flow and PCM collisions (Eqs. 14, 32) and the
Nusselt reading together.

The oracle converges to the benchmark with the grid (Ra = 1e5: +4.5 % at 32^2,
+2.4 % at 48^2, +1.6 % at 64^2, +0.63 % at 128^2); the test runs 48^2 and
64^2.  Copies of the oracle with a mistake planted in their corner treatment
miss the benchmark by 17 % and 2.7 % at 64^2 and fail it.
"""
import json
from pathlib import Path

import pytest

from paper_1701_00702_gb300 import inputs

GOLDEN = json.loads((Path(__file__).parent / "golden" / "de_vahl_davis_1983.json").read_text())
REF = {row["Ra"]: row["Nu_mean"] for row in GOLDEN["rows"]}
# lattice diffusivity per Rayleigh number: the peak velocity stays near 0.05
# (Mach number ~0.09) and the run settles within a few ten thousand steps
K_F = {1e3: 0.2, 1e4: 0.05, 1e5: 0.05}


def steady_nu(oracle_mod, p, library=None, chunk=2000, max_steps=60000, rtol=2e-6):
    """Mean hot-wall Nusselt number once it changes by less than rtol per chunk."""
    o = oracle_mod.Oracle(p, library=library)
    prev = None
    while o.steps < max_steps:
        o.run(chunk)
        nu = o.diag()["nu_hot"]
        if prev is not None and abs(nu - prev) < rtol * abs(nu):
            return nu
        prev = nu
    raise AssertionError(f"no steady state within {max_steps} steps (last Nu {prev})")


@pytest.mark.parametrize("Ra", [1e3, 1e4, 1e5])
def test_mean_hot_wall_nusselt_number_matches_the_benchmark(oracle_mod, Ra):
    nu = steady_nu(oracle_mod, inputs.heated_cavity(64, Ra, k_f=K_F[Ra]))
    assert abs(nu / REF[Ra] - 1.0) < 0.02, (Ra, nu, REF[Ra])


def test_nusselt_number_converges_with_the_grid(oracle_mod):
    e48 = steady_nu(oracle_mod, inputs.heated_cavity(48, 1e5)) / REF[1e5] - 1.0
    e64 = steady_nu(oracle_mod, inputs.heated_cavity(64, 1e5)) / REF[1e5] - 1.0
    assert 0.0 < e64 < e48 < 0.035, (e48, e64)
    assert e48 / e64 > (64 / 48) ** 1.2, (e48, e64)   # at least ~first order toward the benchmark


# Plausible mistakes in the corner treatment of Eq. 52, planted one at a time
# in a copy of the oracle's source: the corner node extrapolates from its
# neighbour along the left/right wall instead of the inward diagonal one, or
# the adiabatic top/bottom wall instead of the left/right wall decides the
# corner's temperature.  (Extrapolating from the neighbour along the
# top/bottom wall is not planted: that wall node's own pull would read past
# the end of the oracle's arrays at one corner.)
MUTANTS = {
    "corner_from_side_wall_neighbour": (
        "pull(c, t, F, G, Hh, x + dx, y + dy, &nf);",
        "pull(c, t, F, G, Hh, x + (dy != 0 ? 0 : dx), y + dy, &nf);"),
    "corner_temperature_from_top_bottom_wall": (
        "int side = wx ? (x == 0 ? 0 : 1) : (y == 0 ? 2 : 3);",
        "int side = (dy != 0) ? (y == 0 ? 2 : 3) : (x == 0 ? 0 : 1);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_a_wrong_corner_treatment_fails_the_benchmark(oracle_mod, tmp_path, name):
    old, new = MUTANTS[name]
    src = (Path(oracle_mod.__file__).parent / "lbm_oracle.c").read_text()
    assert src.count(old) == 1
    mutant = tmp_path / f"lbm_oracle_{name}.c"
    mutant.write_text(src.replace(old, new))
    lib = oracle_mod.load(oracle_mod.build(src=mutant, out=tmp_path / f"liboracle_{name}.so"))
    nu = steady_nu(oracle_mod, inputs.heated_cavity(64, 1e5), library=lib)
    assert abs(nu / REF[1e5] - 1.0) > 0.02, (name, nu)   # the benchmark test above would fail
