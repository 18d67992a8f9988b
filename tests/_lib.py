"""Helpers shared by the tests: build/load the CUDA library on demand."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pfsh.h")


def ensure_built() -> str:
    path = os.path.join(ROOT, "paper_1904_05988_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_pfsh_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def declared_functions() -> list[str]:
    """Names of the functions declared in include/pfsh.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s*([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))
