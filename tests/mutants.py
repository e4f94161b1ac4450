"""Planted mistakes in the oracle, for showing that a pin catches them.

``mutant(edits)`` compiles a copy of ``oracle/lbm_oracle.c`` with textual edits (each
``(old, new)`` pair must match exactly once) into a temporary directory, with the oracle's
own compiler flags, and makes every ``oracle`` call use that copy inside the ``with`` block.
The oracle's source is never modified.
"""
from __future__ import annotations

import contextlib
import os
import subprocess
import tempfile


@contextlib.contextmanager
def mutant(edits):
    import oracle

    src = open(os.path.join(os.path.dirname(oracle.__file__), "lbm_oracle.c")).read()
    for old, new in edits:
        assert src.count(old) == 1, f"edit target not unique in the oracle source: {old!r}"
        src = src.replace(old, new)
    with tempfile.TemporaryDirectory() as tmp:
        c_path = os.path.join(tmp, "lbm_oracle.c")
        with open(c_path, "w") as fh:
            fh.write(src)
        so = os.path.join(tmp, "liboracle_mutant.so")
        inc = os.path.dirname(oracle.__file__)
        subprocess.run(["gcc", *oracle.CFLAGS, "-I", inc, "-o", so, c_path, "-lm"], check=True)
        saved = oracle.lib()
        oracle._lib = oracle.load(so)
        try:
            yield
        finally:
            oracle._lib = saved
