"""Stored expected values: small text fixtures, each naming the passage of the
paper it follows, written by ``make_golden.py`` from the FP64 oracle.

File format (plain text, one fixture per file):

* lines starting with ``#`` are comments (the title and the citation);
* ``@ key value`` sets a scalar (an int, or a string for ``kind``);
* ``[name] d0 d1 ...`` starts an array of that shape, followed by its values,
  whitespace separated, written with ``repr`` so that every float64 reads back
  exactly.

This module only parses the files; it holds no dynamics arithmetic.
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

FIXTURES = (
    "rnea_n7.txt",
    "rnea_n5_moving_base.txt",
    "fd_n6.txt",
    "vjp_n4.txt",
    "mass_matrix_n5.txt",
)


class Fixture:
    def __init__(self, name, header, scalars, arrays):
        self.name = name
        self.header = header
        self.scalars = scalars
        self.arrays = arrays

    def __getitem__(self, key):
        return self.arrays[key]

    def __contains__(self, key):
        return key in self.arrays


def path(name):
    return os.path.join(HERE, name)


def parse(text, name="<text>"):
    header, scalars, arrays = [], {}, {}
    cur, shape, vals = None, None, []

    def close():
        if cur is None:
            return
        count = int(np.prod(shape)) if shape else 1
        if len(vals) != count:
            raise ValueError(f"{name}: array {cur} holds {len(vals)} values, shape wants {count}")
        arrays[cur] = np.array(vals, dtype=np.float64).reshape(shape)

    for line in text.splitlines():
        s = line.strip()
        if not s:
            continue
        if s.startswith("#"):
            header.append(s[1:].strip())
        elif s.startswith("@"):
            _, key, value = s.split(None, 2)
            scalars[key] = int(value) if value.lstrip("-").isdigit() else value
        elif s.startswith("["):
            close()
            head, _, dims = s.partition("]")
            cur, shape, vals = head[1:], tuple(int(d) for d in dims.split()), []
        else:
            if cur is None:
                raise ValueError(f"{name}: values before the first array")
            vals.extend(float(v) for v in s.split())
    close()
    return Fixture(name, header, scalars, arrays)


def load(name):
    with open(path(name)) as f:
        return parse(f.read(), name)


def format_fixture(title, citation, scalars, arrays):
    """Text of a fixture; arrays as (name, ndarray) pairs in order."""
    out = [f"# {title}"]
    out.extend(f"# {c}" for c in citation)
    out.append("# written by tests/golden/make_golden.py from the FP64 oracle")
    for k, v in scalars.items():
        out.append(f"@ {k} {v}")
    for k, a in arrays:
        a = np.asarray(a, dtype=np.float64)
        out.append(f"[{k}] " + " ".join(str(d) for d in a.shape))
        flat = a.reshape(-1, a.shape[-1]) if a.ndim > 1 else a.reshape(1, -1)
        for row in flat:
            out.append(" ".join(repr(float(x)) for x in row))
    return "\n".join(out) + "\n"
