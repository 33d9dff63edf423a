"""Planted mistakes: a copy of the oracle's C sources with one edit, built
into its own library, so that a pin test can show it catches that mistake.
Test infrastructure only (the copy lives in pytest's temporary directory)."""
import os
import shutil

import oracle


def planted_library(tmp_dir, filename: str, old: str, new: str) -> str:
    """Build the oracle with the single occurrence of `old` in `filename`
    replaced by `new`; returns the path of the library."""
    src = os.path.dirname(os.path.abspath(oracle.__file__))
    dst = os.path.join(str(tmp_dir), "planted_src")
    os.makedirs(dst, exist_ok=True)
    for f in os.listdir(src):
        if f.endswith(".c") or f.endswith(".h"):
            shutil.copy(os.path.join(src, f), os.path.join(dst, f))
    path = os.path.join(dst, filename)
    text = open(path).read()
    if text.count(old) != 1:
        raise AssertionError("planted edit must match exactly once in %s: %r" % (filename, old))
    with open(path, "w") as fh:
        fh.write(text.replace(old, new))
    out = os.path.join(str(tmp_dir), "liboracle_planted.so")
    oracle.compile_library(dst, out)
    return out
