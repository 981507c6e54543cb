"""Physics check of the whole model: the double-diffusive cavity of Sec. 3.2 run
to a steady state on the GPU, its average Nusselt and Sherwood numbers compared
with the values the paper prints (tests/golden/ddc_sec3_2_tables.json).

The stop test asks for R < 2e-6; FP32 storage leaves a round-off floor of about
1e-6 on this lattice (limit cycles of the rounded update), so a run that ends at
max_steps with R below 5e-6 counts as steady.  The paper's values are matched to
0.5 % (the grid study of Sec. 3.2 moves them by about 0.1 % between 250 and 350
nodes); the hot and cold wall fluxes agree to 0.5 % (what enters leaves)."""
import json
import os

import pytest

from paper_2101_03055_gb300 import analysis, inputs as I

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ddc_sec3_2_tables.json")))
FLOOR = 5e-6


def steady_cavity(cdf, L, A, Ra, Sr, Df, tol=2e-6, max_steps=4_000_000):
    c = GOLD["common"]
    pb = I.ddc_cavity(L, Ra=Ra, Pr=c["Pr"], Le=c["Le"], Nc=c["Nc"], Df=Df, Sr=Sr, ny=int(round(A * L)))
    s = cdf.Solver(pb)
    ok, steps, R = s.run_to_steady(tol, 5000, max_steps)
    return s.moments(), ok, steps, R


def check(cdf, Ra, A, S, D, Nu_ref, Sh_ref):
    M, ok, steps, R = steady_cavity(cdf, 300, A, Ra, S, D)
    Nu, Sh, _, _ = analysis.nusselt_sherwood(M, D, S)
    Nu_e, Sh_e, _, _ = analysis.nusselt_sherwood(M, D, S, T_wall=0.0, C_wall=0.0, east=True)
    print(f"Ra={Ra:g} A={A:g} S=D={S:g}: steps={steps} R={R:.2e} Nu={Nu:.4f} (paper {Nu_ref}) "
          f"Sh={Sh:.4f} (paper {Sh_ref}) east Nu={Nu_e:.4f} Sh={Sh_e:.4f}")
    assert ok or R < FLOOR, R
    assert abs(Nu - Nu_e) / Nu < 5e-3 and abs(Sh - Sh_e) / Sh < 5e-3
    assert abs(Nu - Nu_ref) / Nu_ref < 5e-3
    assert abs(Sh - Sh_ref) / Sh_ref < 5e-3


def row(table, key):
    return [r for r in GOLD[table]["rows"] if r[0] == key][0][1:]


@pytest.mark.parametrize("Ra", [1e3, 1e4, 1e5])
def test_nusselt_sherwood_vs_rayleigh(cdf, Ra):
    t = GOLD["vs_Ra"]
    check(cdf, Ra, t["A"], t["S_TC"], t["D_CT"], *row("vs_Ra", Ra))


@pytest.mark.parametrize("A", [0.5, 1.0])
def test_nusselt_sherwood_vs_aspect_ratio(cdf, A):
    t = GOLD["vs_A"]
    check(cdf, t["Ra"], A, t["S_TC"], t["D_CT"], *row("vs_A", A))


@pytest.mark.parametrize("SD", [-0.2, 0.0])
def test_nusselt_sherwood_vs_soret_dufour(cdf, SD):
    t = GOLD["vs_S_TC_eq_D_CT"]
    check(cdf, t["Ra"], t["A"], SD, SD, *row("vs_S_TC_eq_D_CT", SD))
