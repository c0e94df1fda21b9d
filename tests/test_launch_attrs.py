"""Static check of the CUDA sources: every kernel launched with a dynamic
shared-memory size that may exceed the 48 KB default gets the opt-in
attribute in the same translation unit.

A template kernel instantiated in several .cu files is a separate function in
each (its host stub has internal linkage), so an attribute set in one file
does not cover a launch in another; such a launch fails once its shared memory
passes 48 KB, which only large problem sizes reach."""
import re
from pathlib import Path

CSRC = Path(__file__).resolve().parent.parent / "paper_1905_09071_gb300" / "csrc"
LAUNCH = re.compile(r"\b(k_\w+)\s*(<[^;{}]*?>)?\s*<<<(.*?)>>>", re.S)
# Dynamic sizes bounded below 48 KB by construction (checked where each is set).
SMALL = {"L.V * sizeof(double)"}  # loss weights: at most 2048 vectors (16 KB)


def split_args(text):
    out, depth, cur = [], 0, ""
    for ch in text:
        if ch in "([<":
            depth += 1
        elif ch in ")]>":
            depth -= 1
        if ch == "," and depth == 0:
            out.append(cur.strip())
            cur = ""
        else:
            cur += ch
    out.append(cur.strip())
    return out


def includes(path, seen):
    for name in re.findall(r'#include "([^"]+)"', path.read_text()):
        p = CSRC / name
        if p.exists() and p not in seen:
            seen.add(p)
            includes(p, seen)
    return seen


def test_split_args_keeps_grid_expressions_whole():
    assert split_args("dim3(a, b), 256, 0, st") == ["dim3(a, b)", "256", "0", "st"]


def test_every_large_dynamic_smem_launch_sets_the_attribute_in_its_own_file():
    units = sorted(CSRC.glob("*.cu"))
    assert units
    missing = []
    for tu in units:
        files = [tu] + sorted(includes(tu, set()))
        launched, allowed = set(), set()
        for f in files:
            text = f.read_text()
            for m in LAUNCH.finditer(text):
                args = split_args(m.group(3))
                if len(args) >= 3 and args[2] not in ("0", "") and args[2] not in SMALL:
                    launched.add(m.group(1))
            allowed.update(re.findall(r"allow_max_smem\(\s*(k_\w+)", text))
        missing += [f"{tu.name}: {k}" for k in sorted(launched - allowed)]
    assert not missing, missing
