"""Compile the oracle's C++ library (test infrastructure; see __init__.py).

``-ffp-contract=off`` is part of the oracle's definition: the vertex stage is
a fixed FP32 operation sequence that must not be fused into FMAs (gcc fuses
by default on aarch64).
"""

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vs_oracle.cpp")
LIB_PATH = os.path.join(HERE, "liboracle.so")

FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
         "-pthread"]


def build_command():
    return ["g++", *FLAGS, SRC, "-o", LIB_PATH]


def build_oracle(check: bool = True):
    tmp = LIB_PATH + ".tmp"
    cmd = build_command()
    cmd[-1] = tmp
    subprocess.run(cmd, check=check)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build_oracle())
