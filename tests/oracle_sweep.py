"""Mutation sweep of the CPU oracle (test infrastructure, CPU only; about half an hour).

Every single-operator change (+ <-> -, < <-> <=, > <-> >=, * -> /) on a code line of the
oracle's time step (contact law, wall geometry, contact search, forces, integration) is
compiled into a copy of the oracle, and the oracle's pins (test_oracle_pins.py,
test_oracle_variants.py, test_golden.py) are run against it in a child process.  A mutant
that every pin passes "survives"; the survivors are the places where the pins do not yet
constrain the oracle, unless the change is equivalent.

    python tests/oracle_sweep.py [first_line last_line] [--jobs N]

Writes one JSON record per mutant to stdout and a summary to stderr; the copies are
compiled under oracle/_build/.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OPS = [(" + ", " - "), (" - ", " + "), (" < ", " <= "), (" <= ", " < "), (" > ", " >= "), (" >= ", " > "),
       (" * ", " / ")]

RUNNER = r"""
import sys, ctypes
sys.path.insert(0, {root!r})
import oracle
oracle._lib = oracle._bind(ctypes.CDLL(sys.argv[1]))
import pytest
sys.exit(int(pytest.main([{pins!r}, {variants!r}, {golden!r}, "-x", "-q", "-p", "no:cacheprovider",
                          "-m", "not gpu"])))
"""


def mutants(lines, first, last):
    out = []
    for ln in range(first - 1, min(last, len(lines))):
        line = lines[ln]
        code = line.split("/*")[0].split("//")[0]
        st = code.strip()
        if not st or st.startswith("#") or st.startswith("*"):
            continue
        for a, b in OPS:
            k = code.find(a)
            while k >= 0:
                out.append((ln + 1, line[:k] + b + line[k + len(a):]))
                k = code.find(a, k + 1)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("first", type=int, nargs="?", default=1)
    ap.add_argument("last", type=int, nargs="?", default=10 ** 9)
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) // 2))
    args = ap.parse_args()
    lines = oracle.source().split("\n")
    build_dir = os.path.join(ROOT, "oracle", "_build")      # the oracle's own (ignored) build folder
    os.makedirs(build_dir, exist_ok=True)
    work = tempfile.mkdtemp(prefix="sweep_", dir=build_dir)
    runner = os.path.join(work, "run_pins.py")
    with open(runner, "w") as f:
        f.write(RUNNER.format(root=ROOT, pins=os.path.join(HERE, "test_oracle_pins.py"),
                              variants=os.path.join(HERE, "test_oracle_variants.py"),
                              golden=os.path.join(HERE, "test_golden.py")))
    todo = mutants(lines, args.first, args.last)

    def run(item):
        idx, (ln, new) = item
        src = list(lines)
        old = src[ln - 1]
        src[ln - 1] = new
        so = os.path.join(work, f"m{idx}.so")
        rec = dict(line=ln, old=old.strip(), new=new.strip())
        try:
            oracle.compile_variant("\n".join(src), so)
        except subprocess.CalledProcessError:
            rec["result"] = "no-compile"
            return rec
        try:
            p = subprocess.run([sys.executable, runner, so], capture_output=True, text=True, timeout=300, cwd=ROOT)
            rec["result"] = "survived" if p.returncode == 0 else "killed"
        except subprocess.TimeoutExpired:
            rec["result"] = "timeout"
        for path in (so, so + ".c"):
            if os.path.exists(path):
                os.remove(path)
        return rec

    counts = {}
    with ThreadPoolExecutor(args.jobs) as pool:
        for rec in pool.map(run, enumerate(todo)):
            counts[rec["result"]] = counts.get(rec["result"], 0) + 1
            print(json.dumps(rec), flush=True)
    os.remove(runner)
    os.rmdir(work)
    print(f"{len(todo)} mutants: {counts}", file=sys.stderr)


if __name__ == "__main__":
    main()
