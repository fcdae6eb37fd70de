"""Mutation check of the oracle's pins (test infrastructure, CPU only).

Each mutant is a copy of cpd_oracle.c with one plausible mistake planted on
one code line: an arithmetic or comparison operator flipped, an off-by-one,
a dropped accumulation, a mode or row index exchanged, the operands of an
index product or an fma swapped, a constant moved. The oracle pins
(tests/test_oracle_pins.py) run against each copy in a temporary directory;
a mutant the pins do not reject is printed as a survivor for inspection
(most survivors are equivalent: loop bounds of free(), symmetric matrices,
branches that compute the same value for block size 1, conditions the
caller repeats). The oracle under oracle/ is never modified.

    python -m oracle.mutants            # both operator sets, all cores
    python -m oracle.mutants --set 1    # one set
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys
import tempfile

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_SRC = os.path.join(_HERE, "cpd_oracle.c")

# (pattern, replacement); replacement None: built from the match's groups
OPERATORS = {
    1: [
        (r"(?<=\s)\+(?=\s)", "-"), (r"(?<=\s)-(?=\s)", "+"),
        (r"(?<=\s)\*(?=\s)", "/"), (r"(?<=\s)/(?=\s)", "*"),
        (r"<=", "<"), (r"(?<![<-])<(?![<=])", "<="),
        (r">=", ">"), (r"(?<![->])>(?![>=])", ">="),
        (r"==", "!="), (r"!=", "=="), (r"&&", "||"), (r"\|\|", "&&"),
        (r"\+=", "-="), (r"-=", "+="), (r"\*=", "/="),
        (r"\+ 1\b", "+ 2"), (r"- 1\b", "- 2"),
        (r"\b0\.5\b", "0.25"), (r"\b1\.0\b", "2.0"),
        (r"\[k\]", "[k ^ 1]"), (r"\[n\]", "[n ^ 1]"), (r"\[r\]", "[r ^ 1]"),
        (r"\(-", "("),
    ],
    2: [
        (r"(?<=\[)(\w+) \* (\w+) \+ (\w+)(?=\])", None),   # a * b + c -> c * b + a
        (r"fma\(([^,()]+), ([^,()]+), ", None),             # fma(x, y, .) -> fma(x, x, .), fma(y, y, .)
        (r"(?<=\[)k(?=\])", "n"), (r"(?<=\[)n(?=\])", "k"), (r"(?<=\[)i(?=\])", "i + 1"),
        (r"\b61\b", "60"), (r"\b40\b", "41"), (r"\b32\b", "16"), (r"\b16\b", "8"),
        (r"\bsqrt\(", "fabs("), (r"\bfloor\(", "ceil("),
        (r"\(double\)t \+", "(double)t + 1.0 +"),
    ],
}


def _code_lines(lines):
    """(index, code) of every line outside comments and preprocessor lines."""
    in_block = False
    for i, line in enumerate(lines):
        s = line.strip()
        if in_block:
            in_block = "*/" not in s
            continue
        if s.startswith("/*"):
            in_block = "*/" not in s
            continue
        if not s or s.startswith("//") or s.startswith("#"):
            continue
        yield i, line.split("/*")[0].split("//")[0]


def mutants(lines, op_set: int):
    out = []
    for i, code in _code_lines(lines):
        for pat, rep in OPERATORS[op_set]:
            for m in re.finditer(pat, code):
                if code[:m.start()].count('"') % 2:
                    continue
                if rep is not None:
                    out.append((i, m.start(), m.end(), rep))
                    continue
                g = m.groups()
                if len(g) == 3:
                    if g[0] != g[2]:
                        out.append((i, m.start(), m.end(), f"{g[2]} * {g[1]} + {g[0]}"))
                else:
                    for v in {g[0], g[1]} if g[0] != g[1] else ():
                        out.append((i, m.start(), m.end(), f"fma({v}, {v}, "))
        if op_set == 1 and re.search(r"(\+=|-=|\*=)", code) and code.rstrip().endswith(";"):
            out.append((i, None, None, None))          # the statement dropped
    return out


def _worker_dir(base: str) -> str:
    w = os.path.join(base, f"w{os.getpid()}")
    if not os.path.exists(w):
        os.makedirs(os.path.join(w, "oracle"))
        os.makedirs(os.path.join(w, "tests"))
        for f in ("__init__.py", "oracle.py"):
            shutil.copy(os.path.join(_HERE, f), os.path.join(w, "oracle"))
        for f in ("conftest.py", "test_oracle_pins.py"):
            shutil.copy(os.path.join(_ROOT, "tests", f), os.path.join(w, "tests"))
        shutil.copytree(os.path.join(_ROOT, "tests", "golden"), os.path.join(w, "tests", "golden"))
    return w


def _run(args):
    base, (i, a, b, rep), lines = args
    w = _worker_dir(base)
    ml = list(lines)
    ml[i] = "/* dropped */\n" if rep is None else ml[i][:a] + rep + ml[i][b:]
    with open(os.path.join(w, "oracle", "cpd_oracle.c"), "w") as f:
        f.write("".join(ml))
    for so in ("liboracle.so", "liboracle_omp.so"):
        p = os.path.join(w, "oracle", so)
        if os.path.exists(p):
            os.remove(p)
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                            "-p", "no:cacheprovider"], cwd=w, capture_output=True, timeout=120)
        txt = (r.stdout + r.stderr).decode(errors="replace")
        status = ("nocompile" if "CalledProcessError" in txt and "gcc" in txt
                  else "survived" if r.returncode == 0 else "killed")
    except subprocess.TimeoutExpired:
        status = "killed"
    return i + 1, lines[i].strip(), ml[i].strip(), status


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--set", type=int, choices=(1, 2), action="append")
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()
    lines = open(_SRC).readlines()
    total = {"killed": 0, "survived": 0, "nocompile": 0}
    with tempfile.TemporaryDirectory(prefix="orc_mutants_") as base:
        for op_set in args.set or (1, 2):
            ms = mutants(lines, op_set)
            with cf.ProcessPoolExecutor(max_workers=args.workers) as ex:
                res = list(ex.map(_run, [(base, m, lines) for m in ms], chunksize=4))
            counts = {k: sum(r[3] == k for r in res) for k in total}
            print(f"set {op_set}: {len(ms)} mutants, " + ", ".join(f"{k} {v}" for k, v in counts.items()))
            for line, old, new, st in res:
                if st == "survived":
                    print(f"  survived L{line}: {old}  ->  {new}")
            for k in total:
                total[k] += counts[k]
    print("total: " + ", ".join(f"{k} {v}" for k, v in total.items()))
    return 0


if __name__ == "__main__":
    sys.exit(main())
