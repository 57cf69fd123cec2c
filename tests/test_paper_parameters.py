"""The parameter presets against the values the paper prints (Sec. IV-B),
stored in tests/golden/paper_parameters.txt.

* params_paper() is the paper's 1/10-scale setup: every printed value, and
  dt = horizon / H (1.2 s over 12 steps).
* params_fullscale() keeps the paper's cost weights (Q, R, S, w_game, the
  four game weights, mu_tail) and scales the distance thresholds s_contest,
  s_role, g_safe and d_col by 5 (the reading of full-size cars; m_bd and the
  vehicle limits are set separately, see the preset's docstring).
"""
import os

import pytest

from paper_2607_25388_b300 import scenario as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            name, *vals = line.split()
            v = [float(x) for x in vals]
            out[name] = v if len(v) > 1 else v[0]
    return out


def test_golden_file_lists_every_printed_value():
    g = _golden()
    assert set(g) == {"K", "H", "horizon_s", "sigma_a", "sigma_delta", "Q", "R", "S", "w_game", "s_contest",
                      "s_role", "mu_tail", "g_safe", "L_IBR", "m_bd", "d_col", "w_contest", "w_long", "w_block",
                      "w_safety"}


def test_paper_preset_is_the_printed_setup():
    g, p = _golden(), S.params_paper()
    for k in ("sigma_a", "sigma_delta", "Q", "R", "S", "w_game", "s_contest", "s_role", "mu_tail", "g_safe",
              "m_bd", "d_col", "w_contest", "w_long", "w_block", "w_safety"):
        assert p[k] == pytest.approx(g[k], rel=0, abs=0), k
    assert p["dt"] == pytest.approx(g["horizon_s"] / g["H"], rel=1e-12)
    assert S.PAPER_SAMPLES == (int(g["K"]), int(g["H"]), int(g["L_IBR"]))


def test_fullscale_preset_keeps_the_weights_and_scales_distances_by_five():
    g, p = _golden(), S.params_fullscale()
    for k in ("Q", "R", "S", "w_game", "w_contest", "w_long", "w_block", "w_safety", "mu_tail"):
        assert p[k] == pytest.approx(g[k], rel=0, abs=0), k
    for k in ("s_contest", "s_role", "g_safe", "d_col"):
        assert p[k] == pytest.approx(5.0 * g[k], rel=1e-12), k
