"""Values printed in the paper, read from the text fixtures under tests/golden/ (each fixture
names the table and section it is taken from)."""

import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table(name):
    """Rows of a fixture as tuples of floats ('#' lines are comments)."""
    rows = []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(tuple(float(x) for x in line.split()))
    return rows
