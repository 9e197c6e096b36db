"""Host-side cost model of the autotuner, pinned to the FLOP row of Table 1.

The printed formulas are read as text from the golden file and evaluated by a
symbolic parser, so a mistyped coefficient in the tuner's model fails here."""
import json
import math
import os

import pytest

from paper_1201_3018_gb300 import tune

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
NAMES = {"full": "full", "symmetric": "sym", "asym2": "asym2", "asym3": "asym3"}


def _eval(expr, N):
    sympy = pytest.importorskip("sympy")
    x = sympy.Symbol("N")
    text = expr.replace("^", "**").replace("log2", "LOG2")
    # implicit products: "4N", ")log", "N+" handled by the parser's transformations
    from sympy.parsing.sympy_parser import (parse_expr, standard_transformations,
                                            implicit_multiplication_application)
    e = parse_expr(text, local_dict={"N": x, "LOG2": lambda a: sympy.log(a, 2)},
                   transformations=standard_transformations + (implicit_multiplication_application,))
    return float(e.subs(x, N))


@pytest.mark.parametrize("domain,key", [("time", "table1_flop_time_domain"), ("freq", "table1_flop_freq_domain")])
@pytest.mark.parametrize("N", [8, 100, 800, 4096])
def test_table1_flops_match_printed(domain, key, N):
    for printed, ours in NAMES.items():
        want = _eval(GOLD[key][printed], N)
        got = tune.table1_flops(ours, domain, N)
        assert got == pytest.approx(want, rel=1e-12), (domain, printed, N)


def test_table1_orderings():
    # Section III: symmetric packing roughly quarters the time-domain work and
    # halves the frequency-domain work; asym M=3 is cheaper than asym M=2
    for N in (100, 800, 4096):
        full = tune.table1_flops("full", "time", N)
        assert full / tune.table1_flops("sym", "time", N) == pytest.approx(4.0, rel=0.02)
        assert tune.table1_flops("asym3", "time", N) < tune.table1_flops("asym2", "time", N) < full
        ff = tune.table1_flops("full", "freq", N)
        assert ff / tune.table1_flops("sym", "freq", N) == pytest.approx(2.0, rel=0.05)


def test_generalised_model_at_table1_block():
    # at W_block = 3N'+1 rounded to a power of two the direct-core model keeps
    # the time-domain ordering of Table 1
    for N in (63, 255, 1023):
        Wb = 1 << math.ceil(math.log2(3 * N + 1))
        f = {m: tune.flops_per_output("direct", N, Wb, m) for m in ("full", "sym", "asym2", "asym3")}
        assert f["sym"] < f["asym3"] < f["asym2"] < f["full"]
        assert tune.flops_per_output("fft", N, Wb, "sym") < tune.flops_per_output("fft", N, Wb, "full")


def test_candidates_respect_geometry():
    for N in (1, 64, 449, 800, 8192):
        cands = tune.candidates(N)
        for core, Wb in cands:
            assert Wb & (Wb - 1) == 0 and Wb - (N | 1) - 1 >= 2
            assert core == "fft" or Wb <= 8192
            if core == "tc":  # the tensor-core core's own limits
                assert (N | 1) <= 449 and Wb % 64 == 0
        assert any(c == "tc" for c, _ in cands) == ((N | 1) <= 449)
        assert not any(c == "tc" for c, _ in tune.candidates(N, pack=0x100))  # per-block selection only
