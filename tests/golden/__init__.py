"""Stored expected values for the CPU pins of the oracle.

Each fixture is a small text file: comment lines (``#``) give the source of
the values, every other line is ``key: value``.  The values come from the
paper (cited by section) or from the published work a reading of the paper
relies on (cited by author and venue); none is produced by this library."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name: str) -> dict:
    """The key: value lines of tests/golden/<name>, values as stripped strings."""
    out = {}
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, value = line.partition(":")
            out[key.strip()] = value.strip()
    return out
