"""Builds the oracle's C code into ``oracle/_build/liboracle.so`` (gcc, -O2).

Test infrastructure only; see ``oracle/__init__.py``.  Portable C: no
architecture flags, so it builds identically on x86_64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "iwpp_oracle.c")
OUT_DIR = os.path.join(_HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")


def build_oracle(force: bool = False, src: str = SRC, out: str = OUT) -> str:
    """Compile ``src`` to the shared library ``out`` if it is missing or stale."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force=True))
