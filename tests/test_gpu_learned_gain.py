"""What the trained proposal gains over the plain sampler at the same sample
budget: a network trained on best responses of the plain planner (73 k
examples from closed-loop ten-car races), evaluated teacher-forced on the
game-on best responses of held-out races.  The learned sampler (2048
proposal + 2048 plain samples) must lower the mean violation of the
responses where neither sampler finds a feasible sample, against 4096 plain
samples; the test prints the whole comparison."""
import json

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_trained_proposal_lowers_violation_at_equal_budget():
    from paper_2607_25388_b300 import learned as LR
    from paper_2607_25388_b300 import scenario as S
    p = S.params_fullscale()
    X, Y = LR.generate_dataset(range(20000, 20060), 20, params=p)
    mlp = LR.Mlp(60, seed=1)
    losses = LR.train(mlp, X, Y, 40, cosine=True)
    assert losses[-1] < 0.2 * losses[0]
    res = LR.compare(mlp, range(200, 203), 3, params=p)
    s = LR.summarize(res)
    print(json.dumps(s))
    assert s["k_match"] == 1.0                       # the standalone plain response reproduces the plan's
    assert s["mean_violation_learned"] < s["mean_violation_plain_eq"]
