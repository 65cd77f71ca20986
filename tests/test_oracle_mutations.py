"""The oracle's pins catch plausible mistakes in the oracle (no GPU).

Each case builds the oracle with one planted mistake (``ORACLE_MUTANT = n``,
planted at the place marked "planted n" in ``oracle/twopaco_oracle.cpp``),
makes the wrappers call that build, and requires the named pins of
``tests/test_oracle.py`` to fail on it. A pin that still passed would not be
checking what it claims to check. The mistakes are the ones a restatement of
the definition most easily makes: a dropped sentinel, an uncomplemented base
on the other strand, inconsistent normalized forms, an off-by-one loop bound
or successor index, a wrong branching threshold, a palindrome's second orientation
forgotten, the sentinel test of Algorithm 1 skipped, a first-pass keep rule
off by one, a class cut that leaves no bins for later classes, an edge length
off by one, and the split definition without sentinels.
"""
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle as O
from oracle import build as oracle_build
from tests import test_oracle as pins

# Brute-force cases of the definition pin: every small k, both strand modes,
# several alphabets (their strings repeat, so sentinel k-mers recur inside).
BRUTE = [c for c in pins._random_cases() if c[1] <= 8]


def _brute(both=None):
    return [(pins.test_definition_matches_brute_force, c) for c in BRUTE
            if both is None or c[2] == both]


MUTANTS = {
    1: ("no sentinels", [(pins.test_fig1_worked_example, (False, 2))]),
    2: ("other strand's predecessor not complemented", _brute(both=True)),
    3: ("k-mers stored under the maximum, looked up under the minimum", _brute(both=True)),
    4: ("last k-mer of a string never flagged", [(pins.test_fig1_worked_example, (False, 2))]),
    5: ("successor read one base early", _brute()),
    6: ("one edge already counts as a branch", [(pins.test_fig1_worked_example, (False, 2))]),
    7: ("a palindrome takes only its forward orientation", _brute(both=True)),
    8: ("Algorithm 1 without its sentinel test", _brute()),
    9: ("first pass keeps a k-mer with one present item", [(pins.test_pass1_sparse_filter_is_exact, ())]),
    10: ("class cut leaves no bin for the later classes", [(pins.test_partition_cuts_examples, ())]),
    11: ("edge length off by one", [(pins.test_edges_are_the_maximal_nonbranching_paths, (3, True))]),
    12: ("split definition without sentinels",
         [(pins.test_parallel_definition_equals_single_thread, (25, True, True))]),
}


@pytest.fixture(scope="module")
def mutant_libs():
    with ThreadPoolExecutor(max_workers=len(MUTANTS)) as ex:
        paths = dict(zip(MUTANTS, ex.map(oracle_build.build_mutant, MUTANTS)))
    return paths


def _fails(pin, args) -> bool:
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


@pytest.mark.parametrize("n", sorted(MUTANTS), ids=[MUTANTS[n][0] for n in sorted(MUTANTS)])
def test_planted_mistake_fails_a_pin(n, mutant_libs):
    what, cases = MUTANTS[n]
    prev = O.use_library(mutant_libs[n])
    try:
        caught = [pin.__name__ for pin, args in cases if _fails(pin, args)]
    finally:
        O.use_library(prev)
    assert caught, f"planted mistake {n} ({what}) passed every pin it should fail"


def test_unplanted_build_passes_the_same_pins():
    """The same pin calls pass on the oracle as built for use."""
    for _, (what, cases) in MUTANTS.items():
        for pin, args in cases:
            assert not _fails(pin, args), (what, pin.__name__, args)
