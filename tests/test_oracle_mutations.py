"""Each planted mistake in the oracle (an off-by-one predicate, the wrong hash
bits, a dropped or sign-flipped term, a reversed tie-break, a wrong join
index, transposed operands, and in the aggregate-first plan a semi-join
taken as a join, a non-strict threshold, a dropped D' or date filter) must
trip at least one pin."""
import pytest

import oracle
import pins

PLANTS = {
    1: "'<' evaluated as '<='",
    2: "partition on the low hash bits",
    3: "revenue drops the (100 - disc) factor",
    4: "revenue uses (100 + disc)",
    5: "top-k tie-break on key descending",
    6: "M.dref looked up off by one",
    7: "group-by with key and value transposed",
    8: "join pair with probe row and build value swapped",
    9: "aggregate-first semi-join counts a key once per M' row",
    10: "aggregate-first threshold compared with >=",
    11: "aggregate-first M' ignores D'",
    12: "aggregate-first aggregation drops the F date filter",
}


@pytest.mark.parametrize("plant", sorted(PLANTS), ids=lambda p: PLANTS[p])
def test_planted_mistake_is_caught(plant):
    failures = []
    oracle.set_plant(plant)
    try:
        for pin in pins.ALL_PINS:
            try:
                pin()
            except AssertionError:
                failures.append(pin.__name__)
    finally:
        oracle.set_plant(0)
    assert failures, f"plant {plant} ({PLANTS[plant]}) passed every pin"
