"""The oracle Boolean against hand-worked per-ray cases of Section 4.1
(slicing, union, intersection, difference with inverted B normals, Figure 6)
and Section 4.1.1 (thin-piece removal): tests/golden/boolean_segments.txt."""
import pytest

import oracle
from golden_cases import cases, expected, ray
from ldni_compare import bit_equal

CASES = cases()


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_oracle_matches_hand_worked_case(case):
    A = ray(case["A"], 1, 1)
    B = ray(case["B"], 100, 2)
    got = oracle.boolean(A, B, case["op"], eps=case["eps"])
    assert bit_equal(got, expected(case, A, B))
