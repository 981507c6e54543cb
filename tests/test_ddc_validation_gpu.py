"""Physics check of the whole model: the double-diffusive cavity of Sec. 3.2 run
to a steady state on the GPU, its average Nusselt and Sherwood numbers compared
with the values the paper prints (tests/golden/ddc_sec3_2_tables.json)."""
import json
import os

import numpy as np
import pytest

from paper_2101_03055_gb300 import analysis, inputs as I

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ddc_sec3_2_tables.json")))


def steady_cavity(cdf, L, A, Ra, Sr, Df, tol=1e-6, max_steps=4_000_000):
    c = GOLD["common"]
    pb = I.ddc_cavity(L, Ra=Ra, Pr=c["Pr"], Le=c["Le"], Nc=c["Nc"], Df=Df, Sr=Sr, ny=int(round(A * L)))
    s = cdf.Solver(pb)
    ok, steps, R = s.run_to_steady(tol, 5000, max_steps)
    return s.moments(), ok, steps, R


@pytest.mark.parametrize("Ra", [1e4, 1e5])
def test_nusselt_sherwood_against_paper_table(cdf, Ra):
    tab = GOLD["vs_Ra"]
    Nu_ref, Sh_ref = [r[1:] for r in tab["rows"] if r[0] == Ra][0]
    M, ok, steps, R = steady_cavity(cdf, 300, tab["A"], Ra, tab["S_TC"], tab["D_CT"])
    Nu, Sh, _, _ = analysis.nusselt_sherwood(M, tab["D_CT"], tab["S_TC"])
    Nu_e, Sh_e, _, _ = analysis.nusselt_sherwood(M, tab["D_CT"], tab["S_TC"], T_wall=0.0, C_wall=0.0, east=True)
    print(f"Ra={Ra:g}: steps={steps} R={R:.2e} Nu={Nu:.4f} (paper {Nu_ref}) Sh={Sh:.4f} (paper {Sh_ref}) "
          f"east Nu={Nu_e:.4f} Sh={Sh_e:.4f}")
    assert ok
    assert abs(Nu - Nu_e) / Nu < 5e-3  # steady: what enters leaves
    assert abs(Nu - Nu_ref) / Nu_ref < 0.02
    assert abs(Sh - Sh_ref) / Sh_ref < 0.02
