"""Shared helpers for the tests of the C-ABI library (no oracle code here)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fr_pcpf.h")


def header_functions():
    """Names of the functions include/fr_pcpf.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", src)))


def ensure_built():
    """Build the library the package loads (the bounds-checked one when the
    environment sets FRP_BOUNDS_CHECK=1)."""
    from paper_2006_10967_gb300 import _capi, build
    return build.build(checked=_capi.CHECKED)
