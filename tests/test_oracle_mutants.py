"""A sample of the oracle mutation sweep, run with the CPU suite: one planted
mistake per oracle module (in a scratch copy, never in the repository) must
make the pins fail.  The full sweep is ``python tests/mutation_sweep.py``."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import mutation_sweep as MS  # noqa: E402

SAMPLE = [
    "append coupling sign",        # krylov.py: Algorithm 2's block matrix
    "X rank1 transposed",          # krylov.py: Eq. A.1
    "pade denominator sign",       # dense.py
    "sketch half order",           # sketch.py
    "philox M0",                   # philox.py
    "grad_t sign",                 # grad.py
    "truth axis order",            # truth.py
]


def test_equivalent_mutants_are_in_the_list():
    labels = {m[3] for m in MS.MUTANTS}
    assert set(MS.EQUIVALENT) <= labels
    assert len(labels) == len(MS.MUTANTS)  # labels are unique


@pytest.mark.parametrize("label", SAMPLE)
def test_planted_mistake_fails_a_pin(label):
    mut = [m for m in MS.MUTANTS if m[3] == label]
    assert len(mut) == 1
    name, status, why = MS.run_one(mut[0])
    assert status == "killed", why


def test_every_mutant_still_applies_to_the_oracle():
    """Each planted edit's pattern occurs exactly once in the current oracle
    source, so a later change to the oracle cannot silently retire a mutant
    from the sweep."""
    stale = []
    for path, old, _new, label in MS.MUTANTS:
        with open(os.path.join(MS.ROOT, path)) as fh:
            if fh.read().count(old) != 1:
                stale.append(label)
    assert not stale, stale
