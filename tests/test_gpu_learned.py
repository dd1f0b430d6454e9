"""What the trained proposer gains over the method without it, and over no extrapolation.

On held-out seeded problems (not in the training set), every mode runs the same number of sweeps
from the same start on the split path; f* is the best fit any mode reaches.  The Section 4.2
rule locks a beta that scales the least-squares fixed point by 1 + beta (1 - alpha) (see the
oracle test of that closed form), so it often stalls short of f*; the committed network proposes
beta per sweep, judged against the rule's sweep from the same checkpoint.

What is asserted, plainly: it reaches f* - 1e-6 on at least as many problems as the rule and in
no more sweeps on average.  Against no extrapolation (beta = 0) it is not faster: it reaches the
target on as many problems within a few sweeps of the same count, and its judged sweeps cost
time, so in seconds it is slower; the test prints both and asserts only that it is not worse
in sweeps by more than 10 %."""
import json

import numpy as np
import pytest

from paper_2503_18759_gb300 import binding as b
from paper_2503_18759_gb300 import learn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_18759_gb300 import build
    build.build()
    b.lib()


def test_trained_proposer_beats_the_rule_on_held_out_problems():
    w = learn.load_weights()
    rows = learn.evaluate(w, learn.problem_set(20000, 10), max_sweeps=60)
    s = learn.summarize(rows)
    print(json.dumps(s))
    assert s["learned"]["reached"] >= s["paper"]["reached"]
    assert s["learned"]["mean_sweeps_to_target"] <= s["paper"]["mean_sweeps_to_target"]
    assert s["learned"]["mean_final_fit"] >= s["paper"]["mean_final_fit"] - 1e-9
    # judged proposals: every accepted one kept the fit from dropping
    assert 0.0 <= s["learned"]["accept_rate"] <= 1.0
    # against beta = 0: no gain in sweeps, and slower in seconds (the judge's second sweeps)
    ln, nn = s["learned"], s["none"]
    print(f"learned vs none: {ln['mean_sweeps_to_target']:.2f} vs {nn['mean_sweeps_to_target']:.2f} sweeps, "
          f"{ln['mean_seconds_to_target'] * 1e3:.2f} vs {nn['mean_seconds_to_target'] * 1e3:.2f} ms, "
          f"reached {ln['reached']} vs {nn['reached']} of {s['problems']}")
    assert ln["reached"] >= nn["reached"] - 1
    assert ln["mean_sweeps_to_target"] <= 1.1 * nn["mean_sweeps_to_target"]
