"""The seeded generators still produce the inputs every workload and measured number is
based on (digests written by tests/golden/make_datagen_digests.py)."""
import json
import os

import pytest

from tests.golden.make_datagen_digests import CASES, digest

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "datagen_digests.json")))


@pytest.mark.parametrize("name", sorted(CASES))
def test_generator_output_is_unchanged(name):
    assert digest(CASES[name]()) == GOLDEN[name], name
