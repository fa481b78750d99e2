"""Load (building first if needed) the CUDA library for the tests."""
import os

from paper_1707_02342_gb300 import build, itmpc

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "itmpc.h")


def load():
    build.build()
    return itmpc.lib()


def header_functions(path=HEADER):
    """Names of the functions declared in a C header (prototypes ending in ');')."""
    import re

    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    names = []
    for m in re.finditer(r"([A-Za-z_][A-Za-z0-9_ \*]*?)\b(itmpc_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text):
        names.append(m.group(2))
    return sorted(set(names))
