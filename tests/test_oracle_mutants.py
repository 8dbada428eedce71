"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each mutant is the oracle's C file compiled with one -DORC_MUTANT=k switch
that plants a plausible error: a dropped neighbour weight on the diagonal,
a flipped sign in b, the wrong gradient plane in a weight, a reversed
gradient residual, a wrong Huber weight, a flipped scale step, a wrong
neighbour index, an inverted CG beta, a residual divided by the variance
instead of the standard deviation, a flipped sign of the x-t coupling in
the joint solve, a stereo variance with the wrong power of the depth step,
a stereo sub-pixel fraction with the wrong sign, a Table II scale fit
with the wrong sign, a Table II scale fit that does not move t, a Huber
warm start one iteration too long, a Huber warm start with the Tukey
threshold.
"""
import pytest

import oracle
import pins

MUTANTS = {
    1: "diag misses wx[i-1]",
    2: "b takes -wx[i-1] gx[i-1]",
    3: "x-weight whitens the y-gradient residual",
    4: "x-gradient residual reversed in the cost",
    5: "Huber weight delta/u^2",
    6: "scale step sign flipped",
    7: "south neighbour indexed i-1",
    8: "CG beta inverted",
    9: "semi residual divided by V",
    10: "joint PCG couples x and t with the wrong sign",
    11: "stereo variance uses |dd| instead of dd^2",
    12: "stereo sub-pixel fraction has the wrong sign",
    13: "Table II fit shifts by mean(x - mu_n)",
    14: "Table II fit leaves t in place",
    15: "Huber warm start runs one GN iteration too long",
    16: "Huber warm start uses the Tukey threshold",
}


@pytest.mark.parametrize("k", sorted(MUTANTS), ids=lambda k: f"m{k}")
def test_mutant_is_caught(k):
    o = oracle.Oracle(oracle.build(mutant=k))
    caught = []
    for pin in pins.ALL:
        try:
            pin(o)
        except (AssertionError, FloatingPointError, ValueError, ZeroDivisionError,
                __import__("numpy").linalg.LinAlgError):
            caught.append(pin.__name__)
    assert caught, f"mutant {k} ({MUTANTS[k]}) passed every pin"
