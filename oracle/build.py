"""Build the CPU oracle (plain C) into oracle/_build/<machine>/liboracle.so.

Test infrastructure: the oracle is compiled here so that tests, the smoke check
and bench.py's CPU baseline can load it; the GPU library never links it.
"""
from __future__ import annotations

import hashlib
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["oracle.c"]
HEADERS = ["oracle.h"]


def build_dir() -> str:
    return os.path.join(HERE, "_build", platform.machine())


def lib_path() -> str:
    return os.path.join(build_dir(), "liboracle.so")


def _digest() -> str:
    h = hashlib.sha256()
    for name in SOURCES + HEADERS:
        with open(os.path.join(HERE, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def compile_sources(src_dir: str, out: str) -> str:
    """Compile oracle.c found in src_dir into the shared library `out`."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
           "-Wall", "-Wextra", "-I", src_dir, "-o", tmp] + [os.path.join(src_dir, s) for s in SOURCES]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle if its sources changed; return the library path."""
    out = lib_path()
    stamp = out + ".sha256"
    digest = _digest()
    if not force and os.path.exists(out) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return out
    compile_sources(HERE, out)
    with open(stamp, "w") as f:
        f.write(digest)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
