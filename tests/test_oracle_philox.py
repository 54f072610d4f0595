"""The oracle's Philox4x32-10 against the published known-answer vectors."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_vectors():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    return np.array(rows, dtype=np.uint64).astype(np.uint32)


def test_oracle_philox_matches_known_answers():
    for row in kat_vectors():
        np.testing.assert_array_equal(oracle.philox(row[:4], row[4:6]), row[6:10])
