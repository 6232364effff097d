"""Values the paper prints, reproduced by the oracle's parameter map
(``tests/golden/paper_values.json`` names the source of each)."""
import json
from pathlib import Path

from paper_1701_00702_gb300 import inputs

GOLDEN = json.loads((Path(__file__).parent / "golden" / "paper_values.json").read_text())


def test_zeta_e_at_section_IVB(oracle_mod):
    g = GOLDEN["zeta_e_sec_IVB"]
    p = inputs.paper_cavity_defaults()
    p.update(g["params"])
    lc = oracle_mod.lattice_config(p)
    assert round(lc["zeta_e"], g["digits"]) == g["value"]


def test_table_I_step_counts(oracle_mod):
    """Fo = t alpha_f / L^2 (Eq. 54) with L = N_x reproduces Table I's step counts."""
    for row in GOLDEN["table_I_steps"]["rows"]:
        p = inputs.paper_cavity_defaults()
        p.update(nx=row["nx"], ny=row["nx"], L_char=float(row["nx"]), Ra=row["Ra"])
        lc = oracle_mod.lattice_config(p)
        steps = row["Fo"] * lc["L"] ** 2 / lc["alpha_f"]
        assert round(steps) == row["steps"]


def test_table_I_rates_are_consistent():
    for row in GOLDEN["table_I_cpu"]["rows"]:
        assert abs(row["steps"] / row["cpu_s"] - row["steps_per_s"]) < 0.01 * row["steps_per_s"]


def test_paper_defaults_respect_remark_I(oracle_mod):
    lc = oracle_mod.lattice_config(inputs.paper_cavity_defaults())
    assert lc["c_fref"] < GOLDEN["stability_cref"]["value"] * lc["c_pl"]
    assert lc["c_mref"] < GOLDEN["stability_cref"]["value"] * lc["c_pm"]
    assert inputs.paper_cavity_defaults()["F_phi"] == GOLDEN["F_phi_metal_foam"]["value"]
