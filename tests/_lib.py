"""Test helper: make sure libhd.so exists (nvcc cross-compiles it on a CPU host)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_buildlib():
    path = os.path.join(ROOT, "paper_2005_05371_gb300", "buildlib.py")
    spec = importlib.util.spec_from_file_location("hd_buildlib", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def ensure_built():
    b = load_buildlib()
    b.build()
    return b.LIB
