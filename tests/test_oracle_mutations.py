"""The pins catch plausible mistakes: each planted mistake in the oracle (a flipped sign, a transposed index, a
dropped reduction, an off-by-one power, a wrong monomial order, a wrong bound) fails at least one pin, while the
oracle itself passes all of them.  Mistakes are compiled into separate library builds (-DQFS_MUTATE=k) and checked
in child processes."""
import json
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
MUTANTS = {
    1: "sign of Delta_1",
    2: "transposed exponents in the splitting u",
    3: "wrong witness monomial",
    4: "lift(g)^p taken mod p instead of mod p^2",
    6: "minus sign of the reduced step",
    7: "f^(p-2) instead of f^(p-1)",
    8: "c^(p-1) subtracted in Algorithm 1",
    9: "products left unreduced",
    10: "ascending instead of descending lex input order",
    11: "zero iterate read as height 1",
    12: "bound tested with < instead of <=",
    14: "t^p subtracted at a transposed lattice point",
}


def run_checks(lib_path):
    r = subprocess.run([sys.executable, os.path.join(HERE, "oracle_pin_checks.py"), lib_path],
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None  # the build crashed: the mistake is caught
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_oracle_passes_every_check():
    res = run_checks(oracle.build())
    assert res is not None and all(res.values()), res


@pytest.mark.parametrize("k", sorted(MUTANTS), ids=[MUTANTS[k] for k in sorted(MUTANTS)])
def test_planted_mistake_is_caught(tmp_path, k):
    path = oracle.build(defines=[f"QFS_MUTATE={k}"], path=str(tmp_path / f"liboracle_m{k}.so"))
    res = run_checks(path)
    assert res is None or not all(res.values()), f"mistake {k} ({MUTANTS[k]}) passed every pin: {res}"
